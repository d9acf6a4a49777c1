// Fused vector kernels of rBiCGStab with one recycle space (Algorithm 4;
// Algorithm 2 when the recycle space is empty), right-preconditioned. The
// scalar recurrences (alpha, omega, beta, rho, the postponed U coefficients
// xi) are advanced on the device by the last block of each
// reduction, so a batch of iterations runs without host synchronisation; a
// device flag stops the remaining kernels of a batch on convergence or
// breakdown.
#include <cmath>
#include <type_traits>
#include "rk_bicg.h"
#include "rk_batch.h"
#include "rk_device.cuh"
#include "rk_df.cuh"

namespace rk {

namespace {

__device__ __forceinline__ bool stopped(const BicgScalars* s) { return s->stop != 0; }

// p = r (first iteration) or p = r + beta (p - omega v)
__device__ __forceinline__ void bicg_p_body(BicgVecs v, BicgScalars* s, int64_t n, int bid, int nblk) {
  if (stopped(s)) return;
  if (s->matvecs >= s->maxmv) {  // the iteration cap (i <= max_itn)
    __syncthreads();
    if (threadIdx.x == 0) {
      s->flag = 3;
      s->stop = 1;
    }
    return;
  }
  const bool first = s->it == 0;
  const double beta = s->beta, omega = s->omega;
  const int64_t stride = (int64_t)nblk * blockDim.x;
  for (int64_t i = (int64_t)bid * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double ri = v.r[i];
    v.p[i] = first ? ri : fma(beta, v.p[i] - omega * v.v[i], ri);
  }
}
__global__ void __launch_bounds__(kRedThreads) k_bicg_p(BicgVecs v, BicgScalars* s, int64_t n) {
  bicg_p_body(v, s, n, blockIdx.x, gridDim.x);
}

// alpha = rho / (r~^T v) after the C projection of v; r~ is orthogonal to C, so r~^T v
// equals r~^T (v - C eta1).
__global__ void k_bicg_alpha(BicgScalars* s, const double* dots, int kc) {
  if (threadIdx.x != 0 || stopped(s)) return;
  s->matvecs += 1;
  const double rtv = dots[kc];
  if (rtv == 0.0 || !isfinite(rtv)) {
    s->flag = 2;
    s->stop = 1;
    return;
  }
  s->alpha = s->rho / rtv;
}

// v <- v - C eta1; s = r - alpha v; ||s||; on convergence the
// half step is recorded (xi += alpha eta1 here, x~ += alpha p
// by k_bicg_half).
template <typename CT>
__device__ __forceinline__ void bicg_s_body(BicgVecs v, BicgScalars* s, int64_t n, int kc,
                                                        const CT* C, int64_t ld, const double* eta1,
                                                        double* xi, double* part, unsigned* counter, int bid, int nblk) {
  if (stopped(s)) return;
  __shared__ double red[32];
  __shared__ int lastflag;
  __shared__ double se[256];
  __shared__ float2 sedf[256];
  for (int q = threadIdx.x; q < kc; q += blockDim.x) {
    se[q] = eta1[q];
    const df e = df_from_double(eta1[q]);
    sedf[q] = make_float2(e.hi, e.lo);
  }
  __syncthreads();
  const double alpha = s->alpha;
  const int64_t stride = (int64_t)nblk * blockDim.x;
  double acc = 0.0;
  for (int64_t i = (int64_t)bid * blockDim.x + threadIdx.x; i < n; i += stride) {
    double vi = v.v[i];
    if (kc) {
      if constexpr (std::is_same<CT, float2>::value) {
        float sh = 0.f, sl = 0.f;  // C eta1 in double-float
        for (int q = 0; q < kc; ++q) {
          const float2 c = __ldg(&C[(int64_t)q * ld + i]);
          df_mac(sh, sl, c.x, c.y, sedf[q].x, sedf[q].y);
        }
        vi = (vi - (double)sh) - (double)sl;
      } else {
        for (int q = 0; q < kc; ++q) vi = fma(-__ldg(&C[(int64_t)q * ld + i]), se[q], vi);  // FP64
      }
      v.v[i] = vi;
    }
    const double si = fma(-alpha, vi, v.r[i]);
    v.s[i] = si;
    acc = fma(si, si, acc);
  }
  const double b = block_sum(acc, red);
  if (threadIdx.x == 0) part[bid] = b;
  if (arrive_last_n(counter, &lastflag, nblk)) {
    reduce_partials(part, nblk, 1, &s->s2);
    __syncthreads();
    if (threadIdx.x == 0) {
      if (sqrt(s->s2) <= s->tolabs) {
        for (int q = 0; q < kc; ++q) xi[q] = fma(alpha, se[q], xi[q]);
        s->half = 1;
        s->flag = 1;
        s->stop = 1;
        s->upd = sqrt(s->s2);
        s->it += 1;
      }
    }
  }
}
template <typename CT>
__global__ void __launch_bounds__(kRedThreads) k_bicg_s(BicgVecs v, BicgScalars* s, int64_t n, int kc,
                                                        const CT* C, int64_t ld, const double* eta1,
                                                        double* xi, double* part, unsigned* counter) {
  bicg_s_body(v, s, n, kc, C, ld, eta1, xi, part, counter, blockIdx.x, gridDim.x);
}

// on convergence at the half step: x~ += alpha p
__global__ void __launch_bounds__(kRedThreads) k_bicg_half(BicgVecs v, BicgScalars* s, int64_t n) {
  if (s->half != 1) return;
  const double alpha = s->alpha;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    v.xt[i] = fma(alpha, v.p[i], v.xt[i]);
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
  }
}

// t <- t - C eta2; omega = t^T s / t^T t (last block).
template <typename CT>
__device__ __forceinline__ void bicg_t_body(BicgVecs v, BicgScalars* s, int64_t n, int kc,
                                                        const CT* C, int64_t ld, const double* eta2,
                                                        double* part, unsigned* counter, int bid, int nblk) {
  if (stopped(s)) return;
  __shared__ double red[32];
  __shared__ int lastflag;
  __shared__ float2 sedf[256];
  __shared__ double se[256];
  for (int q = threadIdx.x; q < kc; q += blockDim.x) {
    se[q] = eta2[q];
    const df e = df_from_double(eta2[q]);
    sedf[q] = make_float2(e.hi, e.lo);
  }
  __syncthreads();
  const int64_t stride = (int64_t)nblk * blockDim.x;
  double ts = 0.0, tt = 0.0;
  for (int64_t i = (int64_t)bid * blockDim.x + threadIdx.x; i < n; i += stride) {
    double ti = v.t[i];
    if (kc) {
      if constexpr (std::is_same<CT, float2>::value) {
        float sh = 0.f, sl = 0.f;  // C eta2 in double-float
        for (int q = 0; q < kc; ++q) {
          const float2 c = __ldg(&C[(int64_t)q * ld + i]);
          df_mac(sh, sl, c.x, c.y, sedf[q].x, sedf[q].y);
        }
        ti = (ti - (double)sh) - (double)sl;
      } else {
        for (int q = 0; q < kc; ++q) ti = fma(-__ldg(&C[(int64_t)q * ld + i]), se[q], ti);  // FP64
      }
      v.t[i] = ti;
    }
    ts = fma(ti, v.s[i], ts);
    tt = fma(ti, ti, tt);
  }
  const double b0 = block_sum(ts, red);
  __syncthreads();
  const double b1 = block_sum(tt, red);
  if (threadIdx.x == 0) {
    part[2 * bid] = b0;
    part[2 * bid + 1] = b1;
  }
  if (arrive_last_n(counter, &lastflag, nblk)) {
    reduce_partials(part, nblk, 2, s->tmp);
    __syncthreads();
    if (threadIdx.x == 0) {
      s->matvecs += 1;
      const double tsv = s->tmp[0], ttv = s->tmp[1];
      if (ttv == 0.0 || !isfinite(ttv)) {
        s->flag = 2;
        s->stop = 1;
      } else {
        s->omega = tsv / ttv;
      }
    }
  }
}
template <typename CT>
__global__ void __launch_bounds__(kRedThreads) k_bicg_t(BicgVecs v, BicgScalars* s, int64_t n, int kc,
                                                        const CT* C, int64_t ld, const double* eta2,
                                                        double* part, unsigned* counter) {
  bicg_t_body(v, s, n, kc, C, ld, eta2, part, counter, blockIdx.x, gridDim.x);
}

// xi += alpha eta1 + omega eta2; x~ += alpha p + omega s;
// r = s - omega t; rho = r~^T r, beta = (rho/rho_old)(alpha/omega); the
// convergence and breakdown tests of the next iteration.
__device__ __forceinline__ void bicg_r_body(BicgVecs v, BicgScalars* s, int64_t n, int kc,
                                                        const double* eta1, const double* eta2, double* xi,
                                                        double* part, unsigned* counter, int bid, int nblk) {
  if (stopped(s)) return;
  __shared__ double red[32];
  __shared__ int lastflag;
  const double alpha = s->alpha, omega = s->omega;
  const int64_t stride = (int64_t)nblk * blockDim.x;
  double rr = 0.0, rtr = 0.0;
  for (int64_t i = (int64_t)bid * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double si = v.s[i];
    v.xt[i] = fma(omega, si, fma(alpha, v.p[i], v.xt[i]));
    const double ri = fma(-omega, v.t[i], si);
    v.r[i] = ri;
    rr = fma(ri, ri, rr);
    rtr = fma(v.rt[i], ri, rtr);
  }
  const double b0 = block_sum(rtr, red);
  __syncthreads();
  const double b1 = block_sum(rr, red);
  if (threadIdx.x == 0) {
    part[2 * bid] = b0;
    part[2 * bid + 1] = b1;
  }
  if (arrive_last_n(counter, &lastflag, nblk)) {
    reduce_partials(part, nblk, 2, s->tmp);
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 0; q < kc; ++q) xi[q] = fma(omega, eta2[q], fma(alpha, eta1[q], xi[q]));
      const double rho_new = s->tmp[0];
      const double rnorm = sqrt(s->tmp[1]);
      s->it += 1;
      s->upd = rnorm;
      if (rnorm <= s->tolabs) {
        s->flag = 1;
        s->stop = 1;
      } else if (omega == 0.0 || fabs(rho_new) <= 1e-14 * s->rtnorm * rnorm || !isfinite(rho_new)) {
        s->flag = 2;
        s->stop = 1;
      } else {
        s->beta = (rho_new / s->rho) * (alpha / omega);
        s->rho = rho_new;
      }
    }
  }
}
__global__ void __launch_bounds__(kRedThreads) k_bicg_r(BicgVecs v, BicgScalars* s, int64_t n, int kc,
                                                        const double* eta1, const double* eta2, double* xi,
                                                        double* part, unsigned* counter) {
  bicg_r_body(v, s, n, kc, eta1, eta2, xi, part, counter, blockIdx.x, gridDim.x);
}

// Start of a pass of Algorithm 4 (after the initial C projection): r~ = r_0, rho = r~^T r_0.
__global__ void k_bicg_init(BicgScalars* s, const double* rho2, double tolabs, int maxmv) {
  if (threadIdx.x != 0) return;
  s->rho = *rho2;
  s->rtnorm = sqrt(*rho2);
  s->tolabs = tolabs;
  s->alpha = s->omega = s->beta = 0.0;
  s->it = 0;
  s->matvecs = 0;
  s->maxmv = maxmv;
  s->half = 0;
  s->upd = sqrt(*rho2);
  const bool conv = sqrt(*rho2) <= tolabs;
  s->flag = conv ? 1 : (maxmv <= 0 ? 3 : 0);
  s->stop = s->flag != 0 ? 1 : 0;
}

// coefficients of the final fold x <- x + M^{-1} x~ - U xi: [-xi; 1]
__global__ void k_bicg_foldcoef(const double* xi, int kc, double* coefv) {
  for (int q = threadIdx.x; q <= kc; q += blockDim.x) coefv[q] = q < kc ? -xi[q] : 1.0;
}

// ---- batched launches: item (i, b) runs block b of problem i's kernel
__global__ void __launch_bounds__(kRedThreads) k_batch_bicg_p(const BatchProb* __restrict__ P,
                                                              const int2* __restrict__ items, int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 w = items[it];
    const BatchProb& q = P[w.x];
    bicg_p_body(q.v, q.bs, q.d.n, w.y, q.nblk);
    __syncthreads();
  }
}

__global__ void k_batch_bicg_alpha(const BatchProb* __restrict__ P, int nprob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nprob) return;
  BicgScalars* s = P[i].bs;
  if (stopped(s)) return;
  // the single-problem k_bicg_alpha, for problem i
  s->matvecs += 1;
  const double rtv = P[i].eta1[P[i].kc];
  if (rtv == 0.0 || !isfinite(rtv)) {
    s->flag = 2;
    s->stop = 1;
    return;
  }
  s->alpha = s->rho / rtv;
}

__global__ void __launch_bounds__(kRedThreads) k_batch_bicg_s(const BatchProb* __restrict__ P,
                                                              const int2* __restrict__ items, int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 w = items[it];
    const BatchProb& q = P[w.x];
    bicg_s_body<double>(q.v, q.bs, q.d.n, q.kc, q.C, q.ld, q.eta1, q.xi, q.part, q.counter, w.y, q.nblk);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kRedThreads) k_batch_bicg_t(const BatchProb* __restrict__ P,
                                                              const int2* __restrict__ items, int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 w = items[it];
    const BatchProb& q = P[w.x];
    bicg_t_body<double>(q.v, q.bs, q.d.n, q.kc, q.C, q.ld, q.eta2, q.part, q.counter, w.y, q.nblk);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kRedThreads) k_batch_bicg_r(const BatchProb* __restrict__ P,
                                                              const int2* __restrict__ items, int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 w = items[it];
    const BatchProb& q = P[w.x];
    bicg_r_body(q.v, q.bs, q.d.n, q.kc, q.eta1, q.eta2, q.xi, q.part, q.counter, w.y, q.nblk);
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_batch_bicg_p(const BatchProb* P, const int2* items, int nitems, int grid, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  k_batch_bicg_p<<<grid < nitems ? grid : nitems, kRedThreads, 0, st>>>(P, items, nitems);
  return cudaGetLastError();
}
cudaError_t launch_batch_bicg_alpha(const BatchProb* P, int nprob, cudaStream_t st) {
  if (nprob <= 0) return cudaSuccess;
  k_batch_bicg_alpha<<<(nprob + 127) / 128, 128, 0, st>>>(P, nprob);
  return cudaGetLastError();
}
cudaError_t launch_batch_bicg_s(const BatchProb* P, const int2* items, int nitems, int grid, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  k_batch_bicg_s<<<grid < nitems ? grid : nitems, kRedThreads, 0, st>>>(P, items, nitems);
  return cudaGetLastError();
}
cudaError_t launch_batch_bicg_t(const BatchProb* P, const int2* items, int nitems, int grid, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  k_batch_bicg_t<<<grid < nitems ? grid : nitems, kRedThreads, 0, st>>>(P, items, nitems);
  return cudaGetLastError();
}
cudaError_t launch_batch_bicg_r(const BatchProb* P, const int2* items, int nitems, int grid, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  k_batch_bicg_r<<<grid < nitems ? grid : nitems, kRedThreads, 0, st>>>(P, items, nitems);
  return cudaGetLastError();
}

cudaError_t launch_bicg_foldcoef(const double* xi, int kc, double* coefv, cudaStream_t st) {
  k_bicg_foldcoef<<<1, 256, 0, st>>>(xi, kc, coefv);
  return cudaGetLastError();
}

cudaError_t launch_bicg_init(BicgScalars* s, const double* rho2, double tolabs, int maxmv, cudaStream_t st) {
  k_bicg_init<<<1, 32, 0, st>>>(s, rho2, tolabs, maxmv);
  return cudaGetLastError();
}

cudaError_t launch_bicg_p(const BicgVecs& v, BicgScalars* s, int64_t n, cudaStream_t st) {
  k_bicg_p<<<red_blocks(n), kRedThreads, 0, st>>>(v, s, n);
  return cudaGetLastError();
}
cudaError_t launch_bicg_alpha(BicgScalars* s, const double* dots, int kc, cudaStream_t st) {
  k_bicg_alpha<<<1, 32, 0, st>>>(s, dots, kc);
  return cudaGetLastError();
}
cudaError_t launch_bicg_s(const BicgVecs& v, BicgScalars* s, int64_t n, int kc, const void* C, bool c_df, int64_t ld,
                          const double* eta1, double* xi, double* part, unsigned* counter, cudaStream_t st) {
  if (c_df)
    k_bicg_s<float2><<<red_blocks(n), kRedThreads, 0, st>>>(v, s, n, kc, (const float2*)C, ld, eta1, xi, part,
                                                            counter);
  else
    k_bicg_s<double><<<red_blocks(n), kRedThreads, 0, st>>>(v, s, n, kc, (const double*)C, ld, eta1, xi, part,
                                                            counter);
  return cudaGetLastError();
}
cudaError_t launch_bicg_half(const BicgVecs& v, BicgScalars* s, int64_t n, cudaStream_t st) {
  k_bicg_half<<<red_blocks(n), kRedThreads, 0, st>>>(v, s, n);
  return cudaGetLastError();
}
cudaError_t launch_bicg_t(const BicgVecs& v, BicgScalars* s, int64_t n, int kc, const void* C, bool c_df, int64_t ld,
                          const double* eta2, double* part, unsigned* counter, cudaStream_t st) {
  if (c_df)
    k_bicg_t<float2><<<red_blocks(n), kRedThreads, 0, st>>>(v, s, n, kc, (const float2*)C, ld, eta2, part, counter);
  else
    k_bicg_t<double><<<red_blocks(n), kRedThreads, 0, st>>>(v, s, n, kc, (const double*)C, ld, eta2, part, counter);
  return cudaGetLastError();
}
cudaError_t launch_bicg_r(const BicgVecs& v, BicgScalars* s, int64_t n, int kc, const double* eta1,
                          const double* eta2, double* xi, double* part, unsigned* counter, cudaStream_t st) {
  k_bicg_r<<<red_blocks(n), kRedThreads, 0, st>>>(v, s, n, kc, eta1, eta2, xi, part, counter);
  return cudaGetLastError();
}

}  // namespace rk
