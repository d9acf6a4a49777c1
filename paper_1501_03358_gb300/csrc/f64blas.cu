// Streaming kernels over the FP64 basis [C V] and U: the block inner
// products of the projections (Algorithms 3 and 4), the orthogonalisation
// update with its fused norm, the row-tiled solution and recycle updates
// (Algorithm 3) and the inner products of the harmonic Ritz problem, with
// FP64 storage and FP64 fused multiply-adds throughout. These are the
// kernels of the RK_FP64 and RK_MIXED precisions; RK_DF runs the
// double-float counterparts of dfblas.cu. Every reduction order is fixed by
// the launch shape, which is a function of n alone (deterministic).
#include "rk_internal.h"
#include "rk_device.cuh"

namespace rk {

namespace {

constexpr int kF64Group = 8;  // columns of Q per block of the fused inner products
constexpr int kWarps = kRedThreads / 32;

// Per-thread values of ncol columns summed over the block in a fixed order
// (warp trees, then the warps in order); results to dst[c] (one write per
// column, by thread c). red: kWarps x 2*kF64Group doubles in shared memory.
__device__ __forceinline__ void block_reduce_cols(const double* vals, int ncol, double (*red)[2 * kF64Group],
                                                  double* dst) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 2 * kF64Group; ++q) {
    if (q < ncol) {
      const double s = warp_sum(vals[q]);
      if (lane == 0) red[wid][q] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x < ncol) {
    double s = red[0][threadIdx.x];
    for (int w = 1; w < kWarps; ++w) s += red[w][threadIdx.x];
    dst[threadIdx.x] = s;
  }
  __syncthreads();
}

// Fused inner products of one delayed-reorthogonalisation Arnoldi step:
// out = [Q^T p (nq), Q^T w (nq), p^T p, p^T w, w^T w]. Grid: x = the column
// groups of kF64Group columns plus one slice for the three scalars, y = row
// ranges of rpb rows. The blocks of one row range are adjacent in launch
// order, so p and w are read from HBM once and from L2 by the other groups.
// A thread keeps 2 x kF64Group FP64 sums; every block writes its partials and
// the last row range of a group to finish sums that group's columns over the
// row ranges (a completion counter per group, fixed order).
// rows [begin, end) of this thread: NC columns' sums with p (vals[q]) and
// with w (vals[kF64Group + q]), one fma each per element, in row order
template <int NC>
__device__ __forceinline__ void dots2_rows(const double* const* col, const double* __restrict__ p,
                                           const double* __restrict__ w, int64_t begin, int64_t end, double* vals) {
  for (int64_t i = begin + threadIdx.x; i < end; i += kRedThreads) {
    const double pv = __ldg(&p[i]), wv = __ldg(&w[i]);
    double v[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) v[q] = __ldg(&col[q][i]);
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      vals[q] = fma(v[q], pv, vals[q]);
      vals[kF64Group + q] = fma(v[q], wv, vals[kF64Group + q]);
    }
  }
}

__global__ void __launch_bounds__(kRedThreads) k_dots2_f64(F64Dots2Args a, int64_t rpb) {
  if (a.skip_flag != nullptr && *a.skip_flag != 0) return;
  __shared__ double red[kWarps][2 * kF64Group];
  __shared__ int lastflag;
  const int ncols = 2 * a.nq + 3;
  const int ngroups = (a.nq + kF64Group - 1) / kF64Group;
  const bool scal = (int)blockIdx.x >= ngroups;
  const int c0 = blockIdx.x * kF64Group;
  const int nc = scal ? 0 : min(kF64Group, a.nq - c0);
  const int64_t begin = (int64_t)blockIdx.y * rpb;
  const int64_t end = min(a.n, begin + rpb);
  double vals[2 * kF64Group];
#pragma unroll
  for (int q = 0; q < 2 * kF64Group; ++q) vals[q] = 0.0;
  if (scal) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int64_t i = begin + threadIdx.x; i < end; i += kRedThreads) {
      const double pv = __ldg(&a.p[i]), wv = __ldg(&a.w[i]);
      s0 = fma(pv, pv, s0);
      s1 = fma(pv, wv, s1);
      s2 = fma(wv, wv, s2);
    }
    vals[0] = s0;
    vals[1] = s1;
    vals[2] = s2;
  } else {
    const double* col[kF64Group];
#pragma unroll
    for (int q = 0; q < kF64Group; ++q) col[q] = a.Q + (int64_t)(c0 + (q < nc ? q : 0)) * a.ld;
    // the group's nc columns as a compile-time count: a last group of fewer
    // than kF64Group columns spends no FP64 fmas on padding
    switch (nc) {
      case 8: dots2_rows<8>(col, a.p, a.w, begin, end, vals); break;
      case 7: dots2_rows<7>(col, a.p, a.w, begin, end, vals); break;
      case 6: dots2_rows<6>(col, a.p, a.w, begin, end, vals); break;
      case 5: dots2_rows<5>(col, a.p, a.w, begin, end, vals); break;
      case 4: dots2_rows<4>(col, a.p, a.w, begin, end, vals); break;
      case 3: dots2_rows<3>(col, a.p, a.w, begin, end, vals); break;
      case 2: dots2_rows<2>(col, a.p, a.w, begin, end, vals); break;
      default: dots2_rows<1>(col, a.p, a.w, begin, end, vals); break;
    }
  }
  // block partials: [Q^T p of the group | Q^T w of the group] or the scalars
  __shared__ double bp[2 * kF64Group];
  if (scal) {
    block_reduce_cols(vals, 3, red, bp);
  } else {
    // pack the w-sums after the nc p-sums
#pragma unroll
    for (int q = 0; q < kF64Group; ++q)
      if (q >= nc) vals[kF64Group + q] = 0.0;
    double packed[2 * kF64Group];
#pragma unroll
    for (int q = 0; q < 2 * kF64Group; ++q) packed[q] = 0.0;
#pragma unroll
    for (int q = 0; q < kF64Group; ++q) {
      packed[q] = vals[q];
      packed[kF64Group + q] = vals[kF64Group + q];
    }
    block_reduce_cols(packed, 2 * kF64Group, red, bp);
  }
  double* prow = a.part + (int64_t)blockIdx.y * ncols;
  if (threadIdx.x == 0) {
    if (scal) {
      prow[2 * a.nq + 0] = bp[0];
      prow[2 * a.nq + 1] = bp[1];
      prow[2 * a.nq + 2] = bp[2];
    } else {
      for (int q = 0; q < nc; ++q) {
        prow[c0 + q] = bp[q];
        prow[a.nq + c0 + q] = bp[kF64Group + q];
      }
    }
  }
  // the last row range of this group sums the group's partials
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(a.counter + blockIdx.x, 1u);
    lastflag = (t == gridDim.y - 1) ? 1 : 0;
  }
  __syncthreads();
  if (lastflag) {
    __threadfence();
    if (threadIdx.x == 0) a.counter[blockIdx.x] = 0u;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nout = scal ? 3 : 2 * nc;
    for (int t = wid; t < nout; t += kWarps) {
      const int c = scal ? 2 * a.nq + t : (t < nc ? c0 + t : a.nq + c0 + (t - nc));
      double sum = 0.0;
      for (int by = lane; by < (int)gridDim.y; by += 32) sum += __ldcg(&a.part[(int64_t)by * ncols + c]);
      sum = warp_sum(sum);
      if (lane == 0) a.out[c] = sum;
    }
  }
}

// R columns q .. q + R - 1 of one row: av += sum Q_qu ca_u, and bv likewise
// with cb when `both`, in column order
template <int R>
__device__ __forceinline__ void upd2_chunk(const double* col, int64_t ld, int q, const double* ca, const double* cb,
                                           bool both, double& av, double& bv) {
  double v[R];
#pragma unroll
  for (int u = 0; u < R; ++u) v[u] = __ldg(col + (int64_t)(q + u) * ld);
#pragma unroll
  for (int u = 0; u < R; ++u) av = fma(v[u], ca[q + u], av);
  if (both) {
#pragma unroll
    for (int u = 0; u < R; ++u) bv = fma(v[u], cb[q + u], bv);
  }
}

// v = (p - Q a) s0 into p; p_next = (w - Q b) s1 - v s2 into w (mode 0), or
// only v (mode 1); anything else: nothing. One read of Q feeds both sums.
__global__ void __launch_bounds__(kRedThreads) k_update2_f64(F64Update2Args a) {
  const int mode = *a.mode;
  if (mode != 0 && mode != 1) return;
  extern __shared__ double cab[];  // -a | -b, each padded to nq8 = round_up(nq, 8) with zeros
  __shared__ double sc[3];
  const int nq8 = (a.nq + 7) & ~7;
  for (int q = threadIdx.x; q < nq8; q += blockDim.x) {
    cab[q] = q < a.nq ? -a.a[q] : 0.0;
    cab[nq8 + q] = (q < a.nq && mode == 0) ? -a.b[q] : 0.0;
  }
  if (threadIdx.x < 3) sc[threadIdx.x] = a.scal[threadIdx.x];
  __syncthreads();
  const double s0 = sc[0], s1 = sc[1], s2 = sc[2];
  const double* ca = cab;
  const double* cb = cab + nq8;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double av = a.p[i];
    double bv = mode == 0 ? a.w[i] : 0.0;
    const double* col = a.Q + i;
    // chunks of 8 columns (every load of a chunk issued before its
    // multiply-adds), then the remaining 1-7 columns as a compile-time count,
    // so no FP64 fma is spent on padding
    int q = 0;
    for (; q + 8 <= a.nq; q += 8) upd2_chunk<8>(col, a.ld, q, ca, cb, mode == 0, av, bv);
    switch (a.nq - q) {
      case 7: upd2_chunk<7>(col, a.ld, q, ca, cb, mode == 0, av, bv); break;
      case 6: upd2_chunk<6>(col, a.ld, q, ca, cb, mode == 0, av, bv); break;
      case 5: upd2_chunk<5>(col, a.ld, q, ca, cb, mode == 0, av, bv); break;
      case 4: upd2_chunk<4>(col, a.ld, q, ca, cb, mode == 0, av, bv); break;
      case 3: upd2_chunk<3>(col, a.ld, q, ca, cb, mode == 0, av, bv); break;
      case 2: upd2_chunk<2>(col, a.ld, q, ca, cb, mode == 0, av, bv); break;
      case 1: upd2_chunk<1>(col, a.ld, q, ca, cb, mode == 0, av, bv); break;
      default: break;
    }
    const double vf = av * s0;
    a.p[i] = vf;
    if (mode == 0) a.w[i] = fma(bv, s1, -vf * s2);
  }
}

// y_out = (y_in - Q c) * scale and ||y_out||^2 (nrm2 nullable).
// scale: 1; *scale_ptr; or 1/sqrt(*scale_ptr) when scale_rsqrt (1 if that
// value is not positive).
__global__ void __launch_bounds__(kRedThreads) k_update_f64(F64UpdateArgs a) {
  if (a.skip_flag != nullptr && *a.skip_flag != 0) return;
  extern __shared__ double cneg[];
  __shared__ double red[32];
  __shared__ int lastflag;
  __shared__ double scs;
  for (int q = threadIdx.x; q < a.nq; q += blockDim.x) cneg[q] = -a.c[q];
  if (threadIdx.x == 0) {
    double s = 1.0;
    if (a.scale_ptr) {
      const double v = *a.scale_ptr;
      s = a.scale_rsqrt ? (v > 0.0 ? rsqrt(v) : 1.0) : v;
    }
    scs = s;
  }
  __syncthreads();
  const double scale = scs;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double nn = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double y = a.yin[i];
    const double* col = a.Q + i;
    int q = 0;
    for (; q + 4 <= a.nq; q += 4) {
      const double v0 = __ldg(col + (int64_t)(q + 0) * a.ld);
      const double v1 = __ldg(col + (int64_t)(q + 1) * a.ld);
      const double v2 = __ldg(col + (int64_t)(q + 2) * a.ld);
      const double v3 = __ldg(col + (int64_t)(q + 3) * a.ld);
      y = fma(v0, cneg[q + 0], y);
      y = fma(v1, cneg[q + 1], y);
      y = fma(v2, cneg[q + 2], y);
      y = fma(v3, cneg[q + 3], y);
    }
    for (; q < a.nq; ++q) y = fma(__ldg(col + (int64_t)q * a.ld), cneg[q], y);
    if (a.scale_ptr) y *= scale;
    a.yout[i] = y;
    nn = fma(y, y, nn);
  }
  if (a.nrm2 == nullptr) return;
  const double b = block_sum(nn, red);
  if (threadIdx.x == 0) a.part[blockIdx.x] = b;
  if (arrive_last(a.counter, &lastflag)) reduce_partials(a.part, gridDim.x, 1, a.nrm2);
}

// Row-tiled X P with X = [A (na cols), diag(bscale) Bm (nb cols)] and P
// (np x nc, column-major, leading dimension np): a block stages a tile of tr
// rows of X and all of P in shared memory; thread (g, r) computes row r for
// output columns g*CB .. g*CB+CB-1. The tile is read completely before any
// output is written, so out may overlap the input columns (the in-place
// recycle updates). The row scale is applied once: acc = bscale_i * sum_B,
// then the A columns are added. accum: out += (else out =).
template <int CB>
__global__ void __launch_bounds__(256) k_gemm_rows_f64(F64GemmArgs a, int tr, int ncp) {
  extern __shared__ double xs64[];  // X: np * tr | PT: np * ncp | SC: tr
  const int np = a.na + a.nb;
  double* X = xs64;
  double* PT = xs64 + (int64_t)np * tr;
  double* SC = PT + (int64_t)np * ncp;
  const int nthr = blockDim.x;
  for (int t = threadIdx.x; t < np * ncp; t += nthr) {
    const int q = t / ncp, c = t - q * ncp;
    PT[t] = c < a.nc ? a.P[(int64_t)c * np + q] : 0.0;
  }
  const int g = threadIdx.x / tr, r = threadIdx.x - g * tr;
  const int c0 = g * CB;
  const int64_t ntiles = (a.n + tr - 1) / tr;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * tr;
    __syncthreads();  // previous tile fully consumed and written
    for (int t = threadIdx.x; t < np * tr; t += nthr) {
      const int q = t / tr, rr = t - q * tr;
      const int64_t i = r0 + rr;
      const double* src = q < a.na ? a.A + (int64_t)q * a.lda : a.Bm + (int64_t)(q - a.na) * a.ldb;
      X[t] = i < a.n ? __ldg(src + i) : 0.0;
    }
    if (a.bscale) {
      for (int rr = threadIdx.x; rr < tr; rr += nthr) {
        const int64_t i = r0 + rr;
        SC[rr] = i < a.n ? __ldg(&a.bscale[i]) : 0.0;
      }
    }
    __syncthreads();
    double acc[CB];
#pragma unroll
    for (int u = 0; u < CB; ++u) acc[u] = 0.0;
    const double* pt = PT + c0;
    for (int q = a.na; q < np; ++q) {
      const double xv = X[q * tr + r];
      const double* pq = pt + (int64_t)q * ncp;
#pragma unroll
      for (int u = 0; u < CB; ++u) acc[u] = fma(xv, pq[u], acc[u]);
    }
    if (a.bscale && a.nb > 0) {
      const double sc = SC[r];
#pragma unroll
      for (int u = 0; u < CB; ++u) acc[u] *= sc;
    }
    for (int q = 0; q < a.na; ++q) {
      const double xv = X[q * tr + r];
      const double* pq = pt + (int64_t)q * ncp;
#pragma unroll
      for (int u = 0; u < CB; ++u) acc[u] = fma(xv, pq[u], acc[u]);
    }
    __syncthreads();  // every thread has read the tile before any output is written
    const int64_t i = r0 + r;
    if (i < a.n) {
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const int c = c0 + u;
        if (c >= a.nc) break;
        double* o = a.out + (int64_t)c * a.ldo + i;
        *o = a.accum ? *o + acc[u] : acc[u];
      }
    }
  }
}

// One output column (x updates): out_i (+)= sum_{q<na} A_q[i] p_q
// + bscale_i sum_{q>=na} B_q[i] p_q, streamed from global memory.
__global__ void __launch_bounds__(kRedThreads) k_gemv_f64(F64GemmArgs a) {
  extern __shared__ double pv64[];
  const int np = a.na + a.nb;
  for (int q = threadIdx.x; q < np; q += blockDim.x) pv64[q] = a.P[q];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double bs = 0.0, as = 0.0;
    int q = 0;
    for (; q + 4 <= a.nb; q += 4) {
      const double v0 = __ldg(a.Bm + (int64_t)(q + 0) * a.ldb + i);
      const double v1 = __ldg(a.Bm + (int64_t)(q + 1) * a.ldb + i);
      const double v2 = __ldg(a.Bm + (int64_t)(q + 2) * a.ldb + i);
      const double v3 = __ldg(a.Bm + (int64_t)(q + 3) * a.ldb + i);
      bs = fma(v0, pv64[a.na + q + 0], bs);
      bs = fma(v1, pv64[a.na + q + 1], bs);
      bs = fma(v2, pv64[a.na + q + 2], bs);
      bs = fma(v3, pv64[a.na + q + 3], bs);
    }
    for (; q < a.nb; ++q) bs = fma(__ldg(a.Bm + (int64_t)q * a.ldb + i), pv64[a.na + q], bs);
    q = 0;
    for (; q + 4 <= a.na; q += 4) {
      const double v0 = __ldg(a.A + (int64_t)(q + 0) * a.lda + i);
      const double v1 = __ldg(a.A + (int64_t)(q + 1) * a.lda + i);
      const double v2 = __ldg(a.A + (int64_t)(q + 2) * a.lda + i);
      const double v3 = __ldg(a.A + (int64_t)(q + 3) * a.lda + i);
      as = fma(v0, pv64[q + 0], as);
      as = fma(v1, pv64[q + 1], as);
      as = fma(v2, pv64[q + 2], as);
      as = fma(v3, pv64[q + 3], as);
    }
    for (; q < a.na; ++q) as = fma(__ldg(a.A + (int64_t)q * a.lda + i), pv64[q], as);
    if (a.bscale && a.nb > 0) bs *= __ldg(&a.bscale[i]);
    const double r = as + bs;
    double* o = a.out + i;
    *o = a.accum ? *o + r : r;
  }
}

// Gram blocks out[q + l*np] = sum_i X_q[i] d[i] U_l[i] (the inner products
// of the harmonic Ritz problem of the recycle update), X = [A, Bm]. Each
// thread owns a 4 x 4 set of (q, l) pairs (strided by the number of sets)
// and a slice of the tile's rows; the tiles are row-major in shared memory
// with odd strides. The slices are summed in shared memory, every block
// writes its partials, and k_reduce_cols_f64 sums them over blocks in a
// fixed order.
constexpr int kGramTR = 64;
__global__ void __launch_bounds__(256) k_gram_f64(F64GramArgs a, int ob0, int nob, int ns, int sx, int sy) {
  extern __shared__ double gs64[];
  const int np = a.na + a.nb;
  const int nbq = (np + 3) / 4;
  double* X = gs64;                        // kGramTR * sx
  double* Y = X + (int64_t)kGramTR * sx;   // kGramTR * sy
  const int slice = threadIdx.x / nob, ob = threadIdx.x - slice * nob;
  const bool active = slice < ns;
  const int obg = ob0 + ob;
  const int nbl = (a.nu + 3) / 4;
  const int qi = obg % nbq, li = obg / nbq;
  double acc[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) acc[t] = 0.0;
  const int64_t ntiles = (a.n + kGramTR - 1) / kGramTR;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * kGramTR;
    __syncthreads();
    for (int t = threadIdx.x; t < np * kGramTR; t += blockDim.x) {
      const int q = t / kGramTR, r = t % kGramTR;
      const double* src = q < a.na ? a.A + (int64_t)q * a.lda : a.Bm + (int64_t)(q - a.na) * a.ldb;
      const int64_t i = r0 + r;
      X[r * sx + q] = i < a.n ? __ldg(src + i) : 0.0;
    }
    for (int t = threadIdx.x; t < a.nu * kGramTR; t += blockDim.x) {
      const int l = t / kGramTR, r = t % kGramTR;
      const int64_t i = r0 + r;
      double u = i < a.n ? __ldg(a.U + (int64_t)l * a.ldu + i) : 0.0;
      if (a.d != nullptr && i < a.n) u *= __ldg(&a.d[i]);
      Y[r * sy + l] = u;
    }
    __syncthreads();
    if (active) {
      for (int r = slice; r < kGramTR; r += ns) {
        double xv[4], yv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          xv[u] = X[r * sx + qi + nbq * u];
          yv[u] = Y[r * sy + li + nbl * u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u * 4 + v] = fma(xv[u], yv[v], acc[u * 4 + v]);
      }
    }
  }
  // sum the slices: reuse the tile storage as [ns][nob][16]
  __syncthreads();
  double* red = gs64;
  if (active) {
#pragma unroll
    for (int t = 0; t < 16; ++t) red[((int64_t)slice * nob + ob) * 16 + t] = acc[t];
  }
  __syncthreads();
  const int total = np * a.nu;
  for (int t = threadIdx.x; t < nob * 16; t += blockDim.x) {
    const int o = t / 16, e = t - o * 16;
    const int og = ob0 + o;
    const int q = og % nbq + nbq * (e / 4), l = og / nbq + nbl * (e % 4);
    if (q >= np || l >= a.nu) continue;
    double s = red[(int64_t)o * 16 + e];
    for (int sl2 = 1; sl2 < ns; ++sl2) s += red[((int64_t)sl2 * nob + o) * 16 + e];
    a.part[(int64_t)blockIdx.x * total + q + (int64_t)l * np] = s;
  }
}

// out[c] = sum_b part[b * ncols + c], one warp per column, fixed order.
__global__ void __launch_bounds__(256) k_reduce_cols_f64(const double* __restrict__ part, int nblocks, int ncols,
                                                         double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= ncols) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += part[(int64_t)b * ncols + c];
  s = warp_sum(s);
  if (lane == 0) out[c] = s;
}

// dst = src * scale over ncols columns (scale: 1, *scale_ptr or
// 1/sqrt(*scale_ptr)); the first basis vector v_1 = r / ||r|| of a cycle.
__global__ void __launch_bounds__(kRedThreads) k_copy_scaled(int64_t n, const double* __restrict__ src,
                                                             double* __restrict__ dst, const double* scale_ptr,
                                                             int scale_rsqrt, int ncols, int64_t lds, int64_t ldd) {
  double scale = 1.0;
  if (scale_ptr) {
    const double v = *scale_ptr;
    scale = scale_rsqrt ? (v > 0.0 ? rsqrt(v) : 1.0) : v;
  }
  for (int c = 0; c < ncols; ++c)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      dst[c * ldd + i] = __ldg(&src[c * lds + i]) * scale;
}

// In-place change of the storage of ncols columns between FP64 and
// double-float (both 8 bytes per element): to_df rounds each value to its
// double-float pair hi = fl32(v), lo = fl32(v - hi); otherwise hi + lo in
// FP64 (exact unless lo lies more than 29 bits below hi's last bit).
__global__ void __launch_bounds__(kRedThreads) k_convert_basis(int64_t n, int ncols, int64_t ld, void* base,
                                                               int to_df) {
  for (int c = 0; c < ncols; ++c)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const int64_t off = (int64_t)c * ld + i;
      if (to_df) {
        const double v = reinterpret_cast<double*>(base)[off];
        const float hi = __double2float_rn(v);
        const float lo = __double2float_rn(v - (double)hi);
        reinterpret_cast<float2*>(base)[off] = make_float2(hi, lo);
      } else {
        const float2 v = reinterpret_cast<float2*>(base)[off];
        reinterpret_cast<double*>(base)[off] = (double)v.x + (double)v.y;
      }
    }
}

}  // namespace

int dots2_f64_rows(int64_t n) {
  // row ranges: a function of n alone (about 4096 rows each, at most 2 per SM)
  int64_t b = (n + 4095) / 4096;
  if (b < 1) b = 1;
  if (b > 2 * kNumSM) b = 2 * kNumSM;
  return (int)b;
}

cudaError_t launch_dots2_f64(const F64Dots2Args& a, cudaStream_t st) {
  if (dots2_tc_supported(a)) return launch_dots2_tc(a, st);
  const int yb = dots2_f64_rows(a.n);
  const int64_t rpb = (a.n + yb - 1) / yb;
  const dim3 grid((a.nq + kF64Group - 1) / kF64Group + 1, yb);
  k_dots2_f64<<<grid, kRedThreads, 0, st>>>(a, rpb);
  return cudaGetLastError();
}

cudaError_t launch_update2_f64(const F64Update2Args& a, cudaStream_t st) {
  const size_t smem = (size_t)(a.nq > 0 ? 2 * ((a.nq + 7) & ~7) : 1) * sizeof(double);
  k_update2_f64<<<red_blocks(a.n), kRedThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_update_f64(const F64UpdateArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)(a.nq > 0 ? a.nq : 1) * sizeof(double);
  k_update_f64<<<red_blocks(a.n), kRedThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int CB>
static cudaError_t gemm_f64_go(const F64GemmArgs& a, int tr, int ncp, int threads, size_t smem, cudaStream_t st) {
  static std::atomic<uint64_t> done{0};
  once_per_device(done, [] {
    cudaFuncSetAttribute(k_gemm_rows_f64<CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  const int64_t ntiles = (a.n + tr - 1) / tr;
  const int64_t cap = (int64_t)kNumSM * 4;
  const int blocks = (int)(ntiles < cap ? ntiles : cap);
  k_gemm_rows_f64<CB><<<blocks, threads, smem, st>>>(a, tr, ncp);
  return cudaGetLastError();
}

cudaError_t launch_gemm_rows_f64(const F64GemmArgs& a, cudaStream_t st) {
  const int np = a.na + a.nb;
  if (np == 0 || a.nc == 0) return cudaSuccess;
  if (a.nc == 1) {
    const size_t smem = (size_t)np * sizeof(double);
    k_gemv_f64<<<red_blocks(a.n), kRedThreads, smem, st>>>(a);
    return cudaGetLastError();
  }
  // column groups of at most 8 columns (a power of two groups), CB the
  // compiled width that covers a group (P padded with zero columns)
  int ncg = 1;
  while (ncg * 8 < a.nc) ncg *= 2;
  int cb = (a.nc + ncg - 1) / ncg;
  cb = cb <= 2 ? 2 : (cb <= 4 ? 4 : 8);
  const int ncp = ncg * cb;
  int tr = 256 / ncg;
  while (tr > 8 && ((size_t)np * tr + (size_t)np * ncp + tr) * sizeof(double) > 200 * 1024) tr /= 2;
  const size_t smem = ((size_t)np * tr + (size_t)np * ncp + tr) * sizeof(double);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  const int threads = ncg * tr;
  switch (cb) {
    case 2: return gemm_f64_go<2>(a, tr, ncp, threads, smem, st);
    case 4: return gemm_f64_go<4>(a, tr, ncp, threads, smem, st);
    default: return gemm_f64_go<8>(a, tr, ncp, threads, smem, st);
  }
}

cudaError_t launch_gram_f64(const F64GramArgs& a, cudaStream_t st) {
  const int np = a.na + a.nb;
  const int total = np * a.nu;
  if (total == 0) return cudaSuccess;
  const int nbq = (np + 3) / 4, nbl = (a.nu + 3) / 4;
  const int nblk = nbq * nbl;
  const int sx = ((np + 3) / 4) * 4 + 1, sy = ((a.nu + 3) / 4) * 4 + 1;
  const size_t tiles = (size_t)kGramTR * (sx + sy) * sizeof(double);
  static std::atomic<uint64_t> done{0};
  once_per_device(done, [] {
    cudaFuncSetAttribute(k_gram_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  const int blocks = gram_blocks(a.n);
  for (int ob0 = 0; ob0 < nblk; ob0 += 256) {
    const int nob = nblk - ob0 < 256 ? nblk - ob0 : 256;
    int ns = 256 / nob;
    if (ns > 8) ns = 8;
    const size_t redb = (size_t)ns * nob * 16 * sizeof(double);
    const size_t smem = tiles > redb ? tiles : redb;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    k_gram_f64<<<blocks, 256, smem, st>>>(a, ob0, nob, ns, sx, sy);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_reduce_cols_f64<<<(total + 7) / 8, 256, 0, st>>>(a.part, blocks, total, a.out);
  return cudaGetLastError();
}

cudaError_t launch_copy_scaled(int64_t n, const double* src, double* dst, const double* scale_ptr, int scale_rsqrt,
                               int ncols, int64_t lds, int64_t ldd, cudaStream_t st) {
  k_copy_scaled<<<red_blocks(n), kRedThreads, 0, st>>>(n, src, dst, scale_ptr, scale_rsqrt, ncols, lds, ldd);
  return cudaGetLastError();
}

cudaError_t launch_convert_basis(int64_t n, int ncols, int64_t ld, void* base, bool to_df, cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
  k_convert_basis<<<red_blocks(n), kRedThreads, 0, st>>>(n, ncols, ld, base, to_df ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace rk
