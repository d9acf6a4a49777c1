// Structured-grid stencil products (7 or 19 bands) with the right point-Jacobi
// preconditioner fused into the operand load.
//
// Operator: the banded "diagonal storage" matrix of Sec. 2.1 ("Data Layout");
// preconditioner: point Jacobi M = diag(A) applied from the right (Sec. 2.1,
// "Preconditioners"). Each CTA owns a 32 x 8 tile of (x, y) columns and
// marches through a chunk of z planes, keeping three consecutive planes of
// z = M^{-1} v (with a one-cell halo) in shared memory, so every operand is
// fetched from HBM once per tile and scaled once. Per output cell the
// arithmetic order is fixed:
//   w = c_0 * z_P;  w = fma(c_s, z_{nb(s)}, w) for s = 1 .. S-1
// (out-of-domain neighbours contribute fma(0, 0, w)).
//
// The same kernels also evaluate the left-preconditioned forms dinv (A v)
// and dinv (b - A v) (Sec. 2.1, left for GMRES-type solvers), and the global
// sweep of the sub-domain Jacobi preconditioner, one damped point-Jacobi
// sweep y = z + omega dinv (r - A z) (ST_JSWEEP), in the same band order.
#include "rk_internal.h"
#include "rk_batch.h"
#include "rk_device.cuh"
#include "rk_df.cuh"

namespace rk {

namespace {

// neighbour coordinate for a halo load: c in [-1, n]; -1 when the plane or
// row lies outside a non-periodic axis (or is never used).
__device__ __forceinline__ int halo_coord(int c, int n, int periodic) {
  if (c >= 0 && c < n) return c;
  if (c == -1) return periodic ? n - 1 : -1;
  if (c == n) return periodic ? 0 : -1;
  return -1;
}

template <typename VT>
__device__ __forceinline__ double ld_val(const VT* p, int64_t q);
template <>
__device__ __forceinline__ double ld_val<double>(const double* p, int64_t q) { return __ldg(&p[q]); }
template <>
__device__ __forceinline__ double ld_val<float2>(const float2* p, int64_t q) { return df_to_double_i(__ldg(&p[q])); }

template <typename YT>
__device__ __forceinline__ void st_val(YT* p, int64_t q, double w);
template <>
__device__ __forceinline__ void st_val<double>(double* p, int64_t q, double w) { p[q] = w; }
template <>
__device__ __forceinline__ void st_val<float2>(float2* p, int64_t q, double w) { p[q] = df_from_double_i(w); }

// One tile of the product (block coordinates bx, by, bz of the 2.5-D grid);
// returns the thread's sum of squares of its outputs when want_norm.
template <int S, int MODE, typename VT, typename YT>
__device__ __forceinline__ double stencil_tile(const Dims& d, const double* __restrict__ coef,
                                               const double* __restrict__ dinv, const VT* __restrict__ v,
                                               const double* __restrict__ b, YT* __restrict__ y, int bx, int by,
                                               int bz, int zchunk, bool want_norm) {
  __shared__ double sz[3][kTY + 2][kTX + 2];
  const int tx = threadIdx.x & (kTX - 1), ty = threadIdx.x / kTX;
  const int x0 = bx * kTX, y0 = by * kTY;
  const int k0 = bz * zchunk;
  const int k1 = min(k0 + zchunk, d.nz);
  const int gi = x0 + tx, gj = y0 + ty;
  const bool active = gi < d.nx && gj < d.ny;
  const int64_t N = d.n;
  const int64_t plane = (int64_t)d.nx * d.ny;

  auto load_plane = [&](int kk, int slot) {
    const int kw = halo_coord(kk, d.nz, d.pz);
    for (int t = threadIdx.x; t < (kTY + 2) * (kTX + 2); t += kTX * kTY) {
      const int ly = t / (kTX + 2), lx = t - ly * (kTX + 2);
      const int xw = halo_coord(x0 + lx - 1, d.nx, d.px);
      const int yw = halo_coord(y0 + ly - 1, d.ny, d.py);
      double val = 0.0;
      if (kw >= 0 && xw >= 0 && yw >= 0) {
        const int64_t q = (int64_t)xw + (int64_t)d.nx * yw + plane * kw;
        if (MODE == ST_PREC)
          val = __dmul_rn(ld_val<VT>(v, q), __ldg(&dinv[q]));
        else
          val = ld_val<VT>(v, q);
      }
      sz[slot][ly][lx] = val;
    }
  };

  double acc2 = 0.0;
  if (k0 < k1) {
    load_plane(k0 - 1, (k0 + 2) % 3);
    load_plane(k0, k0 % 3);
    for (int k = k0; k < k1; ++k) {
      load_plane(k + 1, (k + 1) % 3);
      __syncthreads();
      if (active) {
        const int sc = k % 3, sm = (k + 2) % 3, sp = (k + 1) % 3;
        const int64_t p = (int64_t)gi + (int64_t)d.nx * gj + plane * k;
        const int cx = tx + 1, cy = ty + 1;
        double w = __dmul_rn(__ldg(&coef[p]), sz[sc][cy][cx]);
        w = fma(__ldg(&coef[1 * N + p]), sz[sc][cy][cx - 1], w);
        w = fma(__ldg(&coef[2 * N + p]), sz[sc][cy][cx + 1], w);
        w = fma(__ldg(&coef[3 * N + p]), sz[sc][cy - 1][cx], w);
        w = fma(__ldg(&coef[4 * N + p]), sz[sc][cy + 1][cx], w);
        w = fma(__ldg(&coef[5 * N + p]), sz[sm][cy][cx], w);
        w = fma(__ldg(&coef[6 * N + p]), sz[sp][cy][cx], w);
        if (S == 19) {
          w = fma(__ldg(&coef[7 * N + p]), sz[sc][cy - 1][cx - 1], w);
          w = fma(__ldg(&coef[8 * N + p]), sz[sc][cy - 1][cx + 1], w);
          w = fma(__ldg(&coef[9 * N + p]), sz[sc][cy + 1][cx - 1], w);
          w = fma(__ldg(&coef[10 * N + p]), sz[sc][cy + 1][cx + 1], w);
          w = fma(__ldg(&coef[11 * N + p]), sz[sm][cy][cx - 1], w);
          w = fma(__ldg(&coef[12 * N + p]), sz[sm][cy][cx + 1], w);
          w = fma(__ldg(&coef[13 * N + p]), sz[sp][cy][cx - 1], w);
          w = fma(__ldg(&coef[14 * N + p]), sz[sp][cy][cx + 1], w);
          w = fma(__ldg(&coef[15 * N + p]), sz[sm][cy - 1][cx], w);
          w = fma(__ldg(&coef[16 * N + p]), sz[sm][cy + 1][cx], w);
          w = fma(__ldg(&coef[17 * N + p]), sz[sp][cy - 1][cx], w);
          w = fma(__ldg(&coef[18 * N + p]), sz[sp][cy + 1][cx], w);
        }
        if (MODE == ST_RESID || MODE == ST_LRESID || MODE == ST_JSWEEP) w = __ldg(&b[p]) - w;
        if (MODE == ST_LEFT || MODE == ST_LRESID || MODE == ST_JSWEEP) w = __dmul_rn(w, __ldg(&dinv[p]));
        if (MODE == ST_JSWEEP) w = fma(kSdOmega, w, sz[sc][cy][cx]);
        st_val<YT>(y, p, w);
        if (want_norm) acc2 = fma(w, w, acc2);
      }
      __syncthreads();
    }
  }
  return acc2;
}

template <int S, int MODE, typename VT = double, typename YT = double>
__global__ void __launch_bounds__(kTX* kTY) k_stencil(Dims d, const double* __restrict__ coef,
                                                      const double* __restrict__ dinv,
                                                      const VT* __restrict__ v,
                                                      const double* __restrict__ b, YT* __restrict__ y,
                                                      double* part, unsigned* counter, double* nrm2,
                                                      const int* skip, int zchunk) {
  if (skip != nullptr && *skip != 0) return;
  __shared__ double red[32];
  __shared__ int lastflag;
  const double acc2 = stencil_tile<S, MODE, VT, YT>(d, coef, dinv, v, b, y, blockIdx.x, blockIdx.y, blockIdx.z,
                                                    zchunk, part != nullptr);
  if (part == nullptr) return;
  const double s = block_sum(acc2, red);
  const int nb = gridDim.x * gridDim.y * gridDim.z;
  const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  if (threadIdx.x == 0) part[bid] = s;
  if (arrive_last(counter, &lastflag)) reduce_partials(part, nb, 1, nrm2);
}

// FP32 operator (the mixed-precision inner product A M^{-1} v): coefficients
// and 1/a_pp rounded to FP32 once, z = (float)v * dinv32, FP32 accumulation in
// the same band order, result widened on store. Input and output are
// double-float (the basis) or FP64 (rBiCGStab's vectors).
template <typename VT>
__device__ __forceinline__ float ld_f32(const VT* p, int64_t q);
template <>
__device__ __forceinline__ float ld_f32<double>(const double* p, int64_t q) { return __double2float_rn(__ldg(&p[q])); }
template <>
__device__ __forceinline__ float ld_f32<float2>(const float2* p, int64_t q) { return __ldg(&p[q]).x; }
template <>
__device__ __forceinline__ float ld_f32<float>(const float* p, int64_t q) { return __ldg(&p[q]); }

template <typename YT>
__device__ __forceinline__ void st_f32(YT* p, int64_t q, float w);
template <>
__device__ __forceinline__ void st_f32<double>(double* p, int64_t q, float w) { p[q] = (double)w; }
template <>
__device__ __forceinline__ void st_f32<float2>(float2* p, int64_t q, float w) { p[q] = make_float2(w, 0.f); }
template <>
__device__ __forceinline__ void st_f32<float>(float* p, int64_t q, float w) { p[q] = w; }

// MODE: ST_PREC y = A32 (d32 .* v32); ST_PLAIN y = A32 v32; ST_LEFT
// y = d32 .* (A32 v32) (the product, then one rounded multiplication);
// ST_JSWEEP y = fmaf(omega32, d32 .* (r32 - A32 v32), v32) (the global damped
// sweep of the FP32 sub-domain preconditioner), every step one FP32 rounding
// in the band order of the FP64 kernels.
template <int S, int MODE, typename VT, typename YT, typename RT>
__device__ __forceinline__ void stencil32_tile(const Dims& d, const float* __restrict__ coef,
                                               const float* __restrict__ dinv, const VT* __restrict__ v,
                                               YT* __restrict__ y, int bx, int by, int bz, int zchunk,
                                               const RT* __restrict__ r, float om) {
  __shared__ float sz[3][kTY + 2][kTX + 2];
  const int tx = threadIdx.x & (kTX - 1), ty = threadIdx.x / kTX;
  const int x0 = bx * kTX, y0 = by * kTY;
  const int k0 = bz * zchunk;
  const int k1 = min(k0 + zchunk, d.nz);
  const int gi = x0 + tx, gj = y0 + ty;
  const bool active = gi < d.nx && gj < d.ny;
  const int64_t N = d.n;
  const int64_t plane = (int64_t)d.nx * d.ny;
  auto load_plane = [&](int kk, int slot) {
    const int kw = halo_coord(kk, d.nz, d.pz);
    for (int t = threadIdx.x; t < (kTY + 2) * (kTX + 2); t += kTX * kTY) {
      const int ly = t / (kTX + 2), lx = t - ly * (kTX + 2);
      const int xw = halo_coord(x0 + lx - 1, d.nx, d.px);
      const int yw = halo_coord(y0 + ly - 1, d.ny, d.py);
      float val = 0.f;
      if (kw >= 0 && xw >= 0 && yw >= 0) {
        const int64_t q = (int64_t)xw + (int64_t)d.nx * yw + plane * kw;
        val = ld_f32<VT>(v, q);
        if (MODE == ST_PREC) val = __fmul_rn(val, __ldg(&dinv[q]));
      }
      sz[slot][ly][lx] = val;
    }
  };
  if (k0 >= k1) return;
  load_plane(k0 - 1, (k0 + 2) % 3);
  load_plane(k0, k0 % 3);
  for (int k = k0; k < k1; ++k) {
    load_plane(k + 1, (k + 1) % 3);
    __syncthreads();
    if (active) {
      const int sc = k % 3, sm = (k + 2) % 3, sp = (k + 1) % 3;
      const int64_t p = (int64_t)gi + (int64_t)d.nx * gj + plane * k;
      const int cx = tx + 1, cy = ty + 1;
      float w = __fmul_rn(__ldg(&coef[p]), sz[sc][cy][cx]);
      w = fmaf(__ldg(&coef[1 * N + p]), sz[sc][cy][cx - 1], w);
      w = fmaf(__ldg(&coef[2 * N + p]), sz[sc][cy][cx + 1], w);
      w = fmaf(__ldg(&coef[3 * N + p]), sz[sc][cy - 1][cx], w);
      w = fmaf(__ldg(&coef[4 * N + p]), sz[sc][cy + 1][cx], w);
      w = fmaf(__ldg(&coef[5 * N + p]), sz[sm][cy][cx], w);
      w = fmaf(__ldg(&coef[6 * N + p]), sz[sp][cy][cx], w);
      if (S == 19) {
        w = fmaf(__ldg(&coef[7 * N + p]), sz[sc][cy - 1][cx - 1], w);
        w = fmaf(__ldg(&coef[8 * N + p]), sz[sc][cy - 1][cx + 1], w);
        w = fmaf(__ldg(&coef[9 * N + p]), sz[sc][cy + 1][cx - 1], w);
        w = fmaf(__ldg(&coef[10 * N + p]), sz[sc][cy + 1][cx + 1], w);
        w = fmaf(__ldg(&coef[11 * N + p]), sz[sm][cy][cx - 1], w);
        w = fmaf(__ldg(&coef[12 * N + p]), sz[sm][cy][cx + 1], w);
        w = fmaf(__ldg(&coef[13 * N + p]), sz[sp][cy][cx - 1], w);
        w = fmaf(__ldg(&coef[14 * N + p]), sz[sp][cy][cx + 1], w);
        w = fmaf(__ldg(&coef[15 * N + p]), sz[sm][cy - 1][cx], w);
        w = fmaf(__ldg(&coef[16 * N + p]), sz[sm][cy + 1][cx], w);
        w = fmaf(__ldg(&coef[17 * N + p]), sz[sp][cy - 1][cx], w);
        w = fmaf(__ldg(&coef[18 * N + p]), sz[sp][cy + 1][cx], w);
      }
      if (MODE == ST_JSWEEP) w = __fsub_rn(ld_f32<RT>(r, p), w);
      if (MODE == ST_LEFT || MODE == ST_JSWEEP) w = __fmul_rn(w, __ldg(&dinv[p]));
      if (MODE == ST_JSWEEP) w = fmaf(om, w, sz[sc][cy][cx]);
      st_f32<YT>(y, p, w);
    }
    __syncthreads();
  }
}

template <int S, int MODE, typename VT, typename YT, typename RT>
__global__ void __launch_bounds__(kTX* kTY) k_stencil32(Dims d, const float* __restrict__ coef,
                                                        const float* __restrict__ dinv, const VT* __restrict__ v,
                                                        YT* __restrict__ y, const int* skip, int zchunk,
                                                        const RT* __restrict__ r, float om) {
  if (skip != nullptr && *skip != 0) return;
  stencil32_tile<S, MODE, VT, YT, RT>(d, coef, dinv, v, y, blockIdx.x, blockIdx.y, blockIdx.z, zchunk, r, om);
}

// Double-float operator (the recurrences' products in RK_DF): the bands and
// 1/a_pp rounded once to double-float (about 48 bits), z = v * (1/a_pp) as a
// normalised double-float product, and per output cell the S band products
// summed in the fixed band order with TwoProduct and lazy double-float
// accumulation (renormalised after every 8 bands and at the end). Everything
// runs on the FP32 pipe; the FP64 stencil above is bound by the FP64 issue
// rate of this GPU (about one DFMA per 64 cycles per sub-partition warp), this
// one by HBM.
template <typename VT>
__device__ __forceinline__ float2 ld_df(const VT* p, int64_t q);
template <>
__device__ __forceinline__ float2 ld_df<float2>(const float2* p, int64_t q) { return __ldg(&p[q]); }
template <>
__device__ __forceinline__ float2 ld_df<double>(const double* p, int64_t q) { return df_from_double_i(__ldg(&p[q])); }

template <typename YT>
__device__ __forceinline__ void st_df(YT* p, int64_t q, float2 w);
template <>
__device__ __forceinline__ void st_df<float2>(float2* p, int64_t q, float2 w) { p[q] = w; }
template <>
__device__ __forceinline__ void st_df<double>(double* p, int64_t q, float2 w) { p[q] = df_to_double_i(w); }

template <int S, int MODE, typename VT, typename YT>
__global__ void __launch_bounds__(kTX* kTY) k_stencil_dd(Dims d, const float2* __restrict__ coef,
                                                         const float2* __restrict__ dinv,
                                                         const VT* __restrict__ v, YT* __restrict__ y,
                                                         const int* skip, int zchunk,
                                                         const float2* __restrict__ bv, float2 om) {
  if (skip != nullptr && *skip != 0) return;
  __shared__ float2 sz[3][kTY + 2][kTX + 2];
  const int tx = threadIdx.x & (kTX - 1), ty = threadIdx.x / kTX;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int k0 = blockIdx.z * zchunk;
  const int k1 = min(k0 + zchunk, d.nz);
  const int gi = x0 + tx, gj = y0 + ty;
  const bool active = gi < d.nx && gj < d.ny;
  const int64_t N = d.n;
  const int64_t plane = (int64_t)d.nx * d.ny;
  // The haloed tile has (kTY + 2)(kTX + 2) <= 2 kTX kTY cells: each thread
  // owns at most two, whose in-plane offsets (-1 outside a wall) are fixed.
  static_assert((kTY + 2) * (kTX + 2) <= 2 * kTX * kTY, "two halo cells per thread");
  constexpr int kCells = (kTY + 2) * (kTX + 2);
  int64_t hoff[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int t = threadIdx.x + r * kTX * kTY;
    hoff[r] = -1;
    if (t < kCells) {
      const int ly = t / (kTX + 2), lx = t - ly * (kTX + 2);
      const int xw = halo_coord(x0 + lx - 1, d.nx, d.px);
      const int yw = halo_coord(y0 + ly - 1, d.ny, d.py);
      if (xw >= 0 && yw >= 0) hoff[r] = (int64_t)xw + (int64_t)d.nx * yw;
    }
  }
  // operands of one plane: fetched into registers one plane ahead, so their
  // latency overlaps a whole plane of arithmetic; scaled and stored later
  float2 rv[2], rd[2];
  auto fetch = [&](int kk) {
    const int kw = halo_coord(kk, d.nz, d.pz);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      rv[r] = rd[r] = make_float2(0.f, 0.f);
      if (kw >= 0 && hoff[r] >= 0) {
        const int64_t q = hoff[r] + plane * kw;
        rv[r] = ld_df<VT>(v, q);
        if (MODE == ST_PREC) rd[r] = __ldg(&dinv[q]);
      }
    }
  };
  auto store = [&](int slot) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int t = threadIdx.x + r * kTX * kTY;
      if (t < kCells) (&sz[slot][0][0])[t] = MODE == ST_PREC ? df_mul(rv[r], rd[r]) : rv[r];
    }
  };
  if (k0 >= k1) return;
  fetch(k0 - 1);
  store((k0 + 2) % 3);
  fetch(k0);
  store(k0 % 3);
  fetch(k0 + 1);
  for (int k = k0; k < k1; ++k) {
    // slot (k + 1) % 3 held plane k - 2, last read before the previous barrier
    store((k + 1) % 3);
    if (k + 1 < k1) fetch(k + 2);
    // the first seven bands of this plane are requested before the barrier
    const int64_t p = (int64_t)gi + (int64_t)d.nx * gj + plane * k;
    float2 cf[7];
#pragma unroll
    for (int s = 0; s < 7; ++s) cf[s] = active ? __ldg(&coef[s * N + p]) : make_float2(0.f, 0.f);
    __syncthreads();
    if (active) {
      const int sc = k % 3, sm = (k + 2) % 3, sp = (k + 1) % 3;
      const int cx = tx + 1, cy = ty + 1;
      float s, c;
      {
        const float2 z = sz[sc][cy][cx];
        df_mul_pair(cf[0].x, cf[0].y, z.x, z.y, s, c);
      }
      auto mac = [&](int band, float2 z) {
        const float2 a = band < 7 ? cf[band < 7 ? band : 0] : __ldg(&coef[band * N + p]);
        df_mac_lazy(s, c, a.x, a.y, z.x, z.y);
      };
      mac(1, sz[sc][cy][cx - 1]);
      mac(2, sz[sc][cy][cx + 1]);
      mac(3, sz[sc][cy - 1][cx]);
      mac(4, sz[sc][cy + 1][cx]);
      mac(5, sz[sm][cy][cx]);
      mac(6, sz[sp][cy][cx]);
      if (S == 19) {
        mac(7, sz[sc][cy - 1][cx - 1]);
        df_renorm(s, c);
        mac(8, sz[sc][cy - 1][cx + 1]);
        mac(9, sz[sc][cy + 1][cx - 1]);
        mac(10, sz[sc][cy + 1][cx + 1]);
        mac(11, sz[sm][cy][cx - 1]);
        mac(12, sz[sm][cy][cx + 1]);
        mac(13, sz[sp][cy][cx - 1]);
        mac(14, sz[sp][cy][cx + 1]);
        mac(15, sz[sm][cy - 1][cx]);
        df_renorm(s, c);
        mac(16, sz[sm][cy + 1][cx]);
        mac(17, sz[sp][cy - 1][cx]);
        mac(18, sz[sp][cy + 1][cx]);
      }
      df_renorm(s, c);
      float2 wv = make_float2(s, c);
      if (MODE == ST_LEFT) wv = df_mul(wv, __ldg(&dinv[p]));
      if (MODE == ST_JSWEEP) {
        // z + omega dinv (b - A z), the damped point-Jacobi sweep
        const float2 u = df_mul(__ldg(&dinv[p]), df_sub(__ldg(&bv[p]), wv));
        wv = df_fma(om, u, sz[sc][cy][cx]);
      }
      st_df<YT>(y, p, wv);
    }
    __syncthreads();
  }
}

// FP64 -> double-float rounding of the operator (RK_DF): hi = RN(x),
// lo = RN(x - hi).
__global__ void k_round_df(int64_t n, const double* __restrict__ src, float2* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = df_from_double_i(src[i]);
}

__global__ void k_round_f32(int64_t n, const double* __restrict__ src, float* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __double2float_rn(src[i]);
}

// Grid of (x, y) tiles x z chunks with about per_sm blocks per SM: 3 for the
// FP64 kernel (FP64-issue bound), 4 for the double-float one, which is bound
// by memory latency and bandwidth and needs many blocks' loads in flight
// (5 fit per SM at 48 registers; 4 leaves room for the rounding of the chunk
// count, so the grid still runs as one wave).
void stencil_grid(const Dims& d, dim3& grid, int& zchunk, int per_sm = 3) {
  const int tx = (d.nx + kTX - 1) / kTX, ty = (d.ny + kTY - 1) / kTY;
  const int tiles = tx * ty;
  int nzc = (per_sm * kNumSM + tiles - 1) / tiles;
  if (nzc > d.nz) nzc = d.nz;
  if (nzc < 1) nzc = 1;
  zchunk = (d.nz + nzc - 1) / nzc;
  nzc = (d.nz + zchunk - 1) / zchunk;
  grid = dim3(tx, ty, nzc);
}

// batched A M^{-1} products of rBiCGStab (right point Jacobi): item (i, t)
// is tile t of problem i in that problem's batched tiling; the FP64 or FP32
// operator per problem; the problem's stop flag skips it. Elementwise, so the
// tiling does not change any value.
template <int S>
__global__ void __launch_bounds__(kTX* kTY) k_batch_stencil(const BatchProb* __restrict__ P,
                                                            const int2* __restrict__ tiles, int ntiles, int which) {
  for (int it = blockIdx.x; it < ntiles; it += gridDim.x) {
    const int2 w = tiles[it];
    const BatchProb& q = P[w.x];
    if (q.bs->stop != 0) continue;
    const int bx = w.y % q.gx, by = (w.y / q.gx) % q.gy, bz = w.y / (q.gx * q.gy);
    const double* vin = which == 0 ? q.v.p : q.v.s;
    double* yout = which == 0 ? q.v.v : q.v.t;
    if (q.f32)
      stencil32_tile<S, ST_PREC, double, double, float>(q.d, q.coef32, q.dinv32, vin, yout, bx, by, bz, q.zchunk,
                                                        nullptr, 0.f);
    else
      stencil_tile<S, ST_PREC, double, double>(q.d, q.coef, q.dinv, vin, nullptr, yout, bx, by, bz, q.zchunk, false);
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_batch_stencil(const BatchProb* P, const int2* tiles, int ntiles, int S, int which, int grid,
                                 cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  const int g = grid < ntiles ? grid : ntiles;
  if (S == 7)
    k_batch_stencil<7><<<g, kTX * kTY, 0, st>>>(P, tiles, ntiles, which);
  else
    k_batch_stencil<19><<<g, kTX * kTY, 0, st>>>(P, tiles, ntiles, which);
  return cudaGetLastError();
}

int stencil_blocks(const Dims& d) {
  dim3 g;
  int zc;
  stencil_grid(d, g, zc);
  return (int)(g.x * g.y * g.z);
}

cudaError_t launch_stencil(const Dims& d, int S, int mode, const double* coef, const double* dinv,
                           const double* v, const double* b, double* y, double* part, unsigned* counter,
                           double* nrm2, const int* skip, cudaStream_t st) {
  dim3 grid;
  int zchunk;
  stencil_grid(d, grid, zchunk);
  const dim3 block(kTX * kTY);
#define RK_ST(SS, MM) k_stencil<SS, MM><<<grid, block, 0, st>>>(d, coef, dinv, v, b, y, part, counter, nrm2, skip, zchunk)
#define RK_ST_MODES(SS)                                 \
  if (mode == ST_PREC) RK_ST(SS, ST_PREC);              \
  else if (mode == ST_PLAIN) RK_ST(SS, ST_PLAIN);       \
  else if (mode == ST_RESID) RK_ST(SS, ST_RESID);       \
  else if (mode == ST_LEFT) RK_ST(SS, ST_LEFT);         \
  else RK_ST(SS, ST_LRESID);
  if (S == 7) {
    RK_ST_MODES(7)
  } else {
    RK_ST_MODES(19)
  }
#undef RK_ST_MODES
#undef RK_ST
  return cudaGetLastError();
}

cudaError_t launch_jsweep(const Dims& d, int S, const double* coef, const double* dinv, const double* z,
                          const double* r, void* y, bool y_df, double* part, unsigned* counter, double* nrm2,
                          const int* skip, cudaStream_t st) {
  dim3 grid;
  int zchunk;
  stencil_grid(d, grid, zchunk);
  const dim3 block(kTX * kTY);
#define RK_SJ(SS, YT)                                                                                          \
  k_stencil<SS, ST_JSWEEP, double, YT><<<grid, block, 0, st>>>(d, coef, dinv, z, r, (YT*)y, part, counter, nrm2, \
                                                               skip, zchunk)
  if (S == 7) {
    if (y_df) RK_SJ(7, float2); else RK_SJ(7, double);
  } else {
    if (y_df) RK_SJ(19, float2); else RK_SJ(19, double);
  }
#undef RK_SJ
  return cudaGetLastError();
}

cudaError_t launch_stencil32(const Dims& d, int S, const float* coef32, const float* dinv32, const void* v,
                             bool v_df, void* y, bool y_df, const int* skip, cudaStream_t st) {
  dim3 grid;
  int zchunk;
  stencil_grid(d, grid, zchunk);
  const dim3 block(kTX * kTY);
#define RK_S32(SS, VT, YT)                                                                                   \
  k_stencil32<SS, ST_PREC, VT, YT, float><<<grid, block, 0, st>>>(d, coef32, dinv32, (const VT*)v, (YT*)y, skip, \
                                                                  zchunk, nullptr, 0.f)
#define RK_S32_T(SS)                            \
  if (v_df && y_df) RK_S32(SS, float2, float2); \
  else if (v_df) RK_S32(SS, float2, double);    \
  else if (y_df) RK_S32(SS, double, float2);    \
  else RK_S32(SS, double, double);
  if (S == 7) {
    RK_S32_T(7)
  } else {
    RK_S32_T(19)
  }
#undef RK_S32_T
#undef RK_S32
  return cudaGetLastError();
}

cudaError_t launch_stencil32_ex(const Dims& d, int S, int mode, const float* coef32, const float* dinv32,
                                const void* v, int v_kind, void* y, int y_kind, const float* r32, const int* skip,
                                cudaStream_t st) {
  dim3 grid;
  int zchunk;
  stencil_grid(d, grid, zchunk);
  const dim3 block(kTX * kTY);
  const float om = (float)kSdOmega;
  // kinds: 0 FP64, 1 FP32 (the FP32 scratch vectors of the sub-domain preconditioner)
#define RK_S32X(SS, MM, VT, YT) \
  k_stencil32<SS, MM, VT, YT, float><<<grid, block, 0, st>>>(d, coef32, dinv32, (const VT*)v, (YT*)y, skip, zchunk, r32, om)
#define RK_S32X_T(SS, MM)                                 \
  if (v_kind == 1 && y_kind == 1) RK_S32X(SS, MM, float, float); \
  else if (v_kind == 1) RK_S32X(SS, MM, float, double);       \
  else if (y_kind == 1) RK_S32X(SS, MM, double, float);       \
  else RK_S32X(SS, MM, double, double);
#define RK_S32X_M(SS)                                                  \
  if (mode == ST_PLAIN) { RK_S32X_T(SS, ST_PLAIN) }                     \
  else if (mode == ST_LEFT) { RK_S32X_T(SS, ST_LEFT) }                  \
  else if (mode == ST_JSWEEP) { RK_S32X_T(SS, ST_JSWEEP) }              \
  else { RK_S32X_T(SS, ST_PREC) }
  if (mode == ST_JSWEEP && r32 == nullptr) return cudaErrorInvalidValue;
  if (S == 7) {
    RK_S32X_M(7)
  } else {
    RK_S32X_M(19)
  }
#undef RK_S32X_M
#undef RK_S32X_T
#undef RK_S32X
  return cudaGetLastError();
}

cudaError_t launch_round_f32(int64_t n, const double* src, float* dst, cudaStream_t st) {
  k_round_f32<<<red_blocks(n), kRedThreads, 0, st>>>(n, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_stencil_df(const Dims& d, int S, int mode, const double* coef, const double* dinv,
                              const void* v, bool v_df, void* y, bool y_df, const int* skip, cudaStream_t st) {
  dim3 grid;
  int zchunk;
  stencil_grid(d, grid, zchunk);
  const dim3 block(kTX * kTY);
  if (mode == ST_RESID || mode == ST_LRESID) return cudaErrorInvalidValue;
#define RK_STD(SS, MM, VT, YT)                                                                                  \
  k_stencil<SS, MM, VT, YT><<<grid, block, 0, st>>>(d, coef, dinv, (const VT*)v, nullptr, (YT*)y, nullptr, nullptr, \
                                                    nullptr, skip, zchunk)
#define RK_STD_TYPES(SS, MM)                    \
  if (v_df && y_df) RK_STD(SS, MM, float2, float2); \
  else if (v_df) RK_STD(SS, MM, float2, double);    \
  else if (y_df) RK_STD(SS, MM, double, float2);    \
  else RK_STD(SS, MM, double, double);
  if (S == 7) {
    if (mode == ST_PREC) { RK_STD_TYPES(7, ST_PREC) } else if (mode == ST_LEFT) { RK_STD_TYPES(7, ST_LEFT) } else { RK_STD_TYPES(7, ST_PLAIN) }
  } else {
    if (mode == ST_PREC) { RK_STD_TYPES(19, ST_PREC) } else if (mode == ST_LEFT) { RK_STD_TYPES(19, ST_LEFT) } else { RK_STD_TYPES(19, ST_PLAIN) }
  }
#undef RK_STD_TYPES
#undef RK_STD
  return cudaGetLastError();
}

cudaError_t launch_jsweep_dd(const Dims& d, int S, const float2* coefd, const float2* dinvd, const float2* z,
                             const float2* b, void* y, bool y_df, const int* skip, cudaStream_t st) {
  dim3 grid;
  int zchunk;
  stencil_grid(d, grid, zchunk, 4);
  const dim3 block(kTX * kTY);
  // omega as a double-float pair
  const float oh = (float)kSdOmega;
  const float2 om = make_float2(oh, (float)(kSdOmega - (double)oh));
#define RK_SJD(SS, YT)                                                                                              \
  k_stencil_dd<SS, ST_JSWEEP, float2, YT><<<grid, block, 0, st>>>(d, coefd, dinvd, z, (YT*)y, skip, zchunk, b, om)
  if (S == 7) {
    if (y_df) RK_SJD(7, float2); else RK_SJD(7, double);
  } else {
    if (y_df) RK_SJD(19, float2); else RK_SJD(19, double);
  }
#undef RK_SJD
  return cudaGetLastError();
}

cudaError_t launch_round_df(int64_t n, const double* src, float2* dst, cudaStream_t st) {
  k_round_df<<<red_blocks(n), kRedThreads, 0, st>>>(n, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_stencil_dd(const Dims& d, int S, int mode, const float2* coefd, const float2* dinvd,
                              const void* v, bool v_df, void* y, bool y_df, const int* skip, cudaStream_t st) {
  if (mode != ST_PREC && mode != ST_PLAIN && mode != ST_LEFT) return cudaErrorInvalidValue;
  dim3 grid;
  int zchunk;
  stencil_grid(d, grid, zchunk, 4);
  const dim3 block(kTX * kTY);
#define RK_SDD(SS, MM, VT, YT)                                                                                 \
  k_stencil_dd<SS, MM, VT, YT><<<grid, block, 0, st>>>(d, coefd, dinvd, (const VT*)v, (YT*)y, skip, zchunk, nullptr, \
                                                       make_float2(0.f, 0.f))
#define RK_SDD_TYPES(SS, MM)                         \
  if (v_df && y_df) RK_SDD(SS, MM, float2, float2); \
  else if (v_df) RK_SDD(SS, MM, float2, double);    \
  else if (y_df) RK_SDD(SS, MM, double, float2);    \
  else RK_SDD(SS, MM, double, double);
  if (S == 7) {
    if (mode == ST_PREC) { RK_SDD_TYPES(7, ST_PREC) } else if (mode == ST_LEFT) { RK_SDD_TYPES(7, ST_LEFT) } else { RK_SDD_TYPES(7, ST_PLAIN) }
  } else {
    if (mode == ST_PREC) { RK_SDD_TYPES(19, ST_PREC) } else if (mode == ST_LEFT) { RK_SDD_TYPES(19, ST_LEFT) } else { RK_SDD_TYPES(19, ST_PLAIN) }
  }
#undef RK_SDD_TYPES
#undef RK_SDD
  return cudaGetLastError();
}

}  // namespace rk
