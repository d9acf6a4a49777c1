// Tall-skinny block kernels for the projections and orthogonalisation:
//  - k_dots:   [Q extra w]^T w for a block of columns, one read of each column
//              (Algorithm 3 lines 6a-6c and 7-9 taken as a block: C^T w and
//              V_j^T w; Algorithm 4 lines 1c, 7a, 12a);
//  - k_update: w <- w - Q c with the norm of the result fused in;
//  - k_gemm_rows: row-tiled X P for the solution update (lines 13-13a) and
//              the in-place recycle update C <- W_hat Q, U <- W P (line 14a);
//  - k_gram:   [C V]^T (M U), the inner products of the harmonic Ritz problem.
// All grid reductions are two-stage with an order fixed by n (deterministic).
#include "rk_internal.h"
#include "rk_device.cuh"

namespace rk {

namespace {

constexpr int kDotCols = 16;

__global__ void __launch_bounds__(kRedThreads) k_dots(DotsArgs a) {
  if (a.skip_flag != nullptr && *a.skip_flag != 0) return;
  __shared__ double red[kRedThreads / 32][kDotCols];
  __shared__ int lastflag;
  const int ncols = a.nq + a.ne + a.self;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int c0 = 0; c0 < ncols; c0 += kDotCols) {
    const double* ptr[kDotCols];
#pragma unroll
    for (int q = 0; q < kDotCols; ++q) {
      const int col = c0 + q;
      if (col < a.nq)
        ptr[q] = a.Q + (int64_t)col * a.ld;
      else if (col < a.nq + a.ne)
        ptr[q] = a.extra[col - a.nq];
      else
        ptr[q] = a.w;
    }
    const int nc = min(kDotCols, ncols - c0);
    double acc[kDotCols];
#pragma unroll
    for (int q = 0; q < kDotCols; ++q) acc[q] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
      const double wi = __ldg(&a.w[i]);
#pragma unroll
      for (int q = 0; q < kDotCols; ++q)
        if (q < nc) acc[q] = fma(__ldg(&ptr[q][i]), wi, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kDotCols; ++q) {
      const double s = warp_sum(acc[q]);
      if (lane == 0) red[wid][q] = s;
    }
    __syncthreads();
    if (threadIdx.x < nc) {
      double s = 0.0;
      for (int w = 0; w < kRedThreads / 32; ++w) s += red[w][threadIdx.x];
      a.part[(int64_t)blockIdx.x * ncols + c0 + threadIdx.x] = s;
    }
    __syncthreads();
  }
  if (arrive_last(a.counter, &lastflag)) reduce_partials(a.part, gridDim.x, ncols, a.out);
}

__global__ void __launch_bounds__(kRedThreads) k_update(UpdateArgs a) {
  if (a.skip_flag != nullptr && *a.skip_flag != 0) return;
  extern __shared__ double cs[];
  __shared__ double red[32];
  __shared__ int lastflag;
  for (int q = threadIdx.x; q < a.nq; q += blockDim.x) cs[q] = a.c[q];
  __syncthreads();
  const double* yin = a.yin ? a.yin : a.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double acc2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double yi = yin[i];
    const double* col = a.Q + i;
    int q = 0;
    for (; q + 4 <= a.nq; q += 4) {
      const double q0 = __ldg(col + (int64_t)(q + 0) * a.ld);
      const double q1 = __ldg(col + (int64_t)(q + 1) * a.ld);
      const double q2 = __ldg(col + (int64_t)(q + 2) * a.ld);
      const double q3 = __ldg(col + (int64_t)(q + 3) * a.ld);
      yi = fma(-q0, cs[q + 0], yi);
      yi = fma(-q1, cs[q + 1], yi);
      yi = fma(-q2, cs[q + 2], yi);
      yi = fma(-q3, cs[q + 3], yi);
    }
    for (; q < a.nq; ++q) yi = fma(-__ldg(col + (int64_t)q * a.ld), cs[q], yi);
    a.y[i] = yi;
    acc2 = fma(yi, yi, acc2);
  }
  if (a.nrm2 == nullptr) return;
  const double s = block_sum(acc2, red);
  if (threadIdx.x == 0) a.part[blockIdx.x] = s;
  if (arrive_last(a.counter, &lastflag)) reduce_partials(a.part, gridDim.x, 1, a.nrm2);
}

// Row tile of the small GEMM: smem holds X[q][r] (np x TR); P (np x nc) is
// read through the read-only cache (every thread of a warp reads the same
// entry).
__global__ void __launch_bounds__(256) k_gemm_rows(GemmRowsArgs a, int tr) {
  if (a.skip_flag != nullptr && *a.skip_flag != 0) return;
  extern __shared__ double sm[];
  const int np = a.na + a.nb;
  double* X = sm;  // np * tr
  const double* P = a.P;
  const int64_t ntiles = (a.n + tr - 1) / tr;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * tr;
    __syncthreads();
    for (int t = threadIdx.x; t < np * tr; t += blockDim.x) {
      const int q = t / tr, r = t - q * tr;
      const int64_t i = r0 + r;
      double val = 0.0;
      if (i < a.n) {
        if (q < a.na)
          val = a.A[(int64_t)q * a.lda + i];
        else {
          val = a.Bm[(int64_t)(q - a.na) * a.ldb + i];
          if (a.bscale) val = __dmul_rn(val, __ldg(&a.bscale[i]));
        }
      }
      X[t] = val;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < a.nc * tr; t += blockDim.x) {
      const int c = t / tr, r = t - c * tr;
      const int64_t i = r0 + r;
      if (i >= a.n) continue;
      double acc = 0.0;
      const double* Pc = P + (int64_t)c * np;
      for (int q = 0; q < np; ++q) acc = fma(X[q * tr + r], __ldg(&Pc[q]), acc);
      double* o = a.out + (int64_t)c * a.ldo + i;
      *o = a.accum ? *o + acc : acc;
    }
  }
}

constexpr int kGramPPT = 8;  // (q, l) pairs per thread per pass

__global__ void __launch_bounds__(256) k_gram(GramArgs a, int pair0, int npairs_pass, int tr) {
  extern __shared__ double sm[];
  __shared__ int lastflag;
  const int np = a.na + a.nb;
  double* X = sm;                     // np * tr
  double* Y = sm + (int64_t)np * tr;  // nu * tr   (d .* U)
  double acc[kGramPPT];
  int qq[kGramPPT], ll[kGramPPT];
#pragma unroll
  for (int t = 0; t < kGramPPT; ++t) {
    acc[t] = 0.0;
    const int pr = pair0 + threadIdx.x + t * blockDim.x;
    qq[t] = pr % np;
    ll[t] = pr / np;
  }
  const int pend = pair0 + npairs_pass;
  const int64_t ntiles = (a.n + tr - 1) / tr;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * tr;
    __syncthreads();
    for (int t = threadIdx.x; t < np * tr; t += blockDim.x) {
      const int q = t / tr, r = t - q * tr;
      const int64_t i = r0 + r;
      double val = 0.0;
      if (i < a.n) val = q < a.na ? a.A[(int64_t)q * a.lda + i] : a.Bm[(int64_t)(q - a.na) * a.ldb + i];
      X[t] = val;
    }
    for (int t = threadIdx.x; t < a.nu * tr; t += blockDim.x) {
      const int l = t / tr, r = t - l * tr;
      const int64_t i = r0 + r;
      double uv = 0.0;
      if (i < a.n) {
        uv = a.U[(int64_t)l * a.ldu + i];
        if (a.d != nullptr) uv = __dmul_rn(__ldg(&a.d[i]), uv);
      }
      Y[t] = uv;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kGramPPT; ++t) {
      const int pr = pair0 + threadIdx.x + t * blockDim.x;
      if (pr < pend) {
        const double* xr = X + qq[t] * tr;
        const double* yr = Y + ll[t] * tr;
        double s = acc[t];
        for (int r = 0; r < tr; ++r) s = fma(xr[r], yr[r], s);
        acc[t] = s;
      }
    }
  }
  const int total = np * a.nu;
#pragma unroll
  for (int t = 0; t < kGramPPT; ++t) {
    const int pr = pair0 + threadIdx.x + t * blockDim.x;
    if (pr < pend) a.part[(int64_t)blockIdx.x * total + pr] = acc[t];
  }
  if (arrive_last(a.counter, &lastflag)) {
    // reduce only this pass's pairs
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = pair0 + wid; c < pend; c += nw) {
      double s = 0.0;
      for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(&a.part[(int64_t)b * total + c]);
      s = warp_sum(s);
      if (lane == 0) a.out[c] = s;
    }
  }
}

__global__ void k_copy(int64_t n, const double* __restrict__ src, double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void k_fill(int64_t n, double val, double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = val;
}

int gemm_tile_rows(int np) { return np <= 96 ? 64 : 32; }

}  // namespace

int gram_blocks(int64_t n) {
  int64_t b = (n + 4095) / 4096;
  if (b < 1) b = 1;
  if (b > 2 * kNumSM) b = 2 * kNumSM;
  return (int)b;
}

cudaError_t launch_dots(const DotsArgs& a, cudaStream_t st) {
  k_dots<<<red_blocks(a.n), kRedThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)(a.nq > 0 ? a.nq : 1) * sizeof(double);
  k_update<<<red_blocks(a.n), kRedThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gemm_rows(const GemmRowsArgs& a, cudaStream_t st) {
  const int np = a.na + a.nb;
  if (np == 0 || a.nc == 0) return cudaSuccess;
  const int tr = gemm_tile_rows(np);
  const size_t smem = (size_t)np * tr * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_gemm_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr_set = true;
  }
  int64_t ntiles = (a.n + tr - 1) / tr;
  int blocks = (int)(ntiles < 4 * kNumSM ? ntiles : 4 * kNumSM);
  k_gemm_rows<<<blocks, 256, smem, st>>>(a, tr);
  return cudaGetLastError();
}

cudaError_t launch_gram(const GramArgs& a, cudaStream_t st) {
  const int np = a.na + a.nb;
  const int total = np * a.nu;
  if (total == 0) return cudaSuccess;
  const int tr = 32;
  const size_t smem = ((size_t)np * tr + (size_t)a.nu * tr) * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr_set = true;
  }
  const int per_pass = 256 * kGramPPT;
  const int blocks = gram_blocks(a.n);
  for (int p0 = 0; p0 < total; p0 += per_pass) {
    const int np_pass = total - p0 < per_pass ? total - p0 : per_pass;
    k_gram<<<blocks, 256, smem, st>>>(a, p0, np_pass, tr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_copy(int64_t n, const double* src, double* dst, cudaStream_t st) {
  k_copy<<<red_blocks(n), kRedThreads, 0, st>>>(n, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_fill(int64_t n, double val, double* dst, cudaStream_t st) {
  k_fill<<<red_blocks(n), kRedThreads, 0, st>>>(n, val, dst);
  return cudaGetLastError();
}

}  // namespace rk
