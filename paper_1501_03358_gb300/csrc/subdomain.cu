// The sub-domain Jacobi preconditioner of Sec. 2.1 ("Preconditioners"): the
// grid is cut into boxes of kSdBX x kSdBY x kSdBZ owned cells; each box,
// grown by kSdOverlap cells on every side (wrapping on periodic axes, cut at
// non-periodic faces), carries the local problem A_ii z_i = r_i (A restricted
// to the grown box: couplings to cells outside it are dropped), solved
// inexactly by kSdSweeps damped Jacobi sweeps from z_i = 0. Each box keeps the
// values of its own cells (restricted additive Schwarz); one damped
// point-Jacobi sweep on the whole grid (the ST_JSWEEP stencil mode) follows.
//
// Every update of a grown-box cell e (global cell p) is evaluated as
//   s = a_0(p) z_e;  s = fma(a_t(p), z_nb(e,t), s)  for t = 1 .. S-1;
//   u = dinv_p (r_p - s);  z_e <- fma(omega, u, z_e)
// with neighbours outside the grown box or the grid read as zero (a finite
// band times zero adds nothing). The first sweep starts from zero, where this
// reduces to z_e = omega (dinv_p r_p).
//
// One CTA per box; both sweep buffers of the grown box live in shared memory
// with a ring of zeros around them, so neighbour reads need no bounds tests.
// The bands, r and 1/a_pp are read from global memory (they stay in L1/L2
// across the sweeps); the kernel is bound by the FP64 pipe, not by HBM.
#include <mutex>

#include "rk_internal.h"
#include "rk_device.cuh"
#include "rk_df.cuh"

namespace rk {

namespace {

constexpr int kEX = kSdBX + 2 * kSdOverlap;  // largest grown box
constexpr int kEY = kSdBY + 2 * kSdOverlap;
constexpr int kEZ = kSdBZ + 2 * kSdOverlap;
constexpr int kPX = kEX + 2;  // with the ring of zeros
constexpr int kPY = kEY + 2;
constexpr int kPZ = kEZ + 2;
constexpr int kPXY = kPX * kPY;
constexpr int kPad = kPXY * kPZ;
constexpr int kSdThreads = 256;
constexpr int kCellsPer = (kEX * kEY * kEZ + kSdThreads - 1) / kSdThreads;
static_assert(kSdSweeps >= 2, "the first and the last sweep are peeled");

// coordinate of a grown-box cell along one axis; -1 beyond a non-periodic face
__device__ __forceinline__ int sd_wrap(int c, int n, int periodic) {
  if (c >= 0 && c < n) return c;
  if (!periodic) return -1;
  return c < 0 ? c + n : c - n;
}

// s = A_ii z at the grown-box cell with padded shared index q (global cell p),
// bands in storage order
template <int S>
__device__ __forceinline__ double sd_row(const double* __restrict__ coef, int64_t N, int64_t p,
                                         const double* z, int q) {
  double s = __dmul_rn(__ldg(&coef[p]), z[q]);
  s = fma(__ldg(&coef[1 * N + p]), z[q - 1], s);
  s = fma(__ldg(&coef[2 * N + p]), z[q + 1], s);
  s = fma(__ldg(&coef[3 * N + p]), z[q - kPX], s);
  s = fma(__ldg(&coef[4 * N + p]), z[q + kPX], s);
  s = fma(__ldg(&coef[5 * N + p]), z[q - kPXY], s);
  s = fma(__ldg(&coef[6 * N + p]), z[q + kPXY], s);
  if (S == 19) {
    s = fma(__ldg(&coef[7 * N + p]), z[q - 1 - kPX], s);
    s = fma(__ldg(&coef[8 * N + p]), z[q + 1 - kPX], s);
    s = fma(__ldg(&coef[9 * N + p]), z[q - 1 + kPX], s);
    s = fma(__ldg(&coef[10 * N + p]), z[q + 1 + kPX], s);
    s = fma(__ldg(&coef[11 * N + p]), z[q - 1 - kPXY], s);
    s = fma(__ldg(&coef[12 * N + p]), z[q + 1 - kPXY], s);
    s = fma(__ldg(&coef[13 * N + p]), z[q - 1 + kPXY], s);
    s = fma(__ldg(&coef[14 * N + p]), z[q + 1 + kPXY], s);
    s = fma(__ldg(&coef[15 * N + p]), z[q - kPX - kPXY], s);
    s = fma(__ldg(&coef[16 * N + p]), z[q + kPX - kPXY], s);
    s = fma(__ldg(&coef[17 * N + p]), z[q - kPX + kPXY], s);
    s = fma(__ldg(&coef[18 * N + p]), z[q + kPX + kPXY], s);
  }
  return s;
}

template <int S>
__global__ void __launch_bounds__(kSdThreads, 2)
    k_subdomain_local(Dims d, const double* __restrict__ coef, const double* __restrict__ dinv,
                      const double* __restrict__ r, double* __restrict__ z, const int* skip, int nbx, int nby) {
  if (skip != nullptr && *skip != 0) return;
  __shared__ double buf[2][kPad];
  const int box = blockIdx.x;
  const int x0 = (box % nbx) * kSdBX, y0 = ((box / nbx) % nby) * kSdBY, z0 = (box / (nbx * nby)) * kSdBZ;
  const int wx = min(kSdBX, d.nx - x0), wy = min(kSdBY, d.ny - y0), wz = min(kSdBZ, d.nz - z0);
  const int ex = wx + 2 * kSdOverlap, ey = wy + 2 * kSdOverlap, ez = wz + 2 * kSdOverlap;
  const int ne = ex * ey * ez;
  const int64_t N = d.n;
  const int64_t plane = (int64_t)d.nx * d.ny;
  for (int t = threadIdx.x; t < 2 * kPad; t += kSdThreads) (&buf[0][0])[t] = 0.0;

  // this thread's grown-box cells: global index (-1 outside the grid), padded
  // shared index, r and 1/a_pp
  int64_t gp[kCellsPer];
  int pe[kCellsPer];
  double rv[kCellsPer], dv[kCellsPer];
#pragma unroll
  for (int i = 0; i < kCellsPer; ++i) {
    const int e = threadIdx.x + i * kSdThreads;
    gp[i] = -1;
    pe[i] = 0;
    rv[i] = 0.0;
    dv[i] = 0.0;
    if (e < ne) {
      const int a = e % ex, b = (e / ex) % ey, c = e / (ex * ey);
      pe[i] = (a + 1) + kPX * ((b + 1) + kPY * (c + 1));
      const int gi = sd_wrap(x0 - kSdOverlap + a, d.nx, d.px);
      const int gj = sd_wrap(y0 - kSdOverlap + b, d.ny, d.py);
      const int gk = sd_wrap(z0 - kSdOverlap + c, d.nz, d.pz);
      if (gi >= 0 && gj >= 0 && gk >= 0) {
        gp[i] = (int64_t)gi + (int64_t)d.nx * gj + plane * gk;
        rv[i] = __ldg(&r[gp[i]]);
        dv[i] = __ldg(&dinv[gp[i]]);
      }
    }
  }
  __syncthreads();
  // sweep 1 from z = 0
#pragma unroll
  for (int i = 0; i < kCellsPer; ++i)
    if (gp[i] >= 0) buf[0][pe[i]] = __dmul_rn(kSdOmega, __dmul_rn(dv[i], rv[i]));
  __syncthreads();
  // sweeps 2 .. kSdSweeps-1 over the whole grown box
  int cur = 0;
  for (int sw = 1; sw < kSdSweeps - 1; ++sw) {
    const double* za = buf[cur];
    double* zb = buf[cur ^ 1];
#pragma unroll
    for (int i = 0; i < kCellsPer; ++i) {
      if (gp[i] < 0) continue;
      const double s = sd_row<S>(coef, N, gp[i], za, pe[i]);
      const double u = __dmul_rn(dv[i], rv[i] - s);
      zb[pe[i]] = fma(kSdOmega, u, za[pe[i]]);
    }
    __syncthreads();
    cur ^= 1;
  }
  // the last sweep on the box's own cells only, written to z
  const double* za = buf[cur];
  const int nown = wx * wy * wz;
  for (int e = threadIdx.x; e < nown; e += kSdThreads) {
    const int a = e % wx, b = (e / wx) % wy, c = e / (wx * wy);
    const int64_t p = (int64_t)(x0 + a) + (int64_t)d.nx * (y0 + b) + plane * (z0 + c);
    const int q = (a + 1 + kSdOverlap) + kPX * ((b + 1 + kSdOverlap) + kPY * (c + 1 + kSdOverlap));
    const double s = sd_row<S>(coef, N, p, za, q);
    const double u = __dmul_rn(__ldg(&dinv[p]), __ldg(&r[p]) - s);
    z[p] = fma(kSdOmega, u, za[q]);
  }
}

// ---- the FP32 variant (the mixed precision, RK_MIXED): the same sweeps with
// the FP32 copies of the bands and of 1/a_pp (each rounded once from FP64),
// r rounded to FP32, omega = RN32(2/3), the sweep buffers in FP32 and every
// operation an FP32 one in the order of the FP64 kernel:
//   s = a_0 z_e; s = fmaf(a_t, z_nb, s); u = d (r - s); z_e <- fmaf(omega, u, z_e)
// (the first sweep omega (d r)). Half the shared memory of the FP64 kernel,
// so 4 CTAs of 256 threads fit an SM.
template <typename RT>
__device__ __forceinline__ float sd_ld32(const RT* p, int64_t q);
template <>
__device__ __forceinline__ float sd_ld32<double>(const double* p, int64_t q) { return __double2float_rn(__ldg(&p[q])); }
template <>
__device__ __forceinline__ float sd_ld32<float>(const float* p, int64_t q) { return __ldg(&p[q]); }

template <int S>
__device__ __forceinline__ float sd_row32(const float* __restrict__ coef, int64_t N, int64_t p, const float* z, int q) {
  float s = __fmul_rn(__ldg(&coef[p]), z[q]);
  s = fmaf(__ldg(&coef[1 * N + p]), z[q - 1], s);
  s = fmaf(__ldg(&coef[2 * N + p]), z[q + 1], s);
  s = fmaf(__ldg(&coef[3 * N + p]), z[q - kPX], s);
  s = fmaf(__ldg(&coef[4 * N + p]), z[q + kPX], s);
  s = fmaf(__ldg(&coef[5 * N + p]), z[q - kPXY], s);
  s = fmaf(__ldg(&coef[6 * N + p]), z[q + kPXY], s);
  if (S == 19) {
    s = fmaf(__ldg(&coef[7 * N + p]), z[q - 1 - kPX], s);
    s = fmaf(__ldg(&coef[8 * N + p]), z[q + 1 - kPX], s);
    s = fmaf(__ldg(&coef[9 * N + p]), z[q - 1 + kPX], s);
    s = fmaf(__ldg(&coef[10 * N + p]), z[q + 1 + kPX], s);
    s = fmaf(__ldg(&coef[11 * N + p]), z[q - 1 - kPXY], s);
    s = fmaf(__ldg(&coef[12 * N + p]), z[q + 1 - kPXY], s);
    s = fmaf(__ldg(&coef[13 * N + p]), z[q - 1 + kPXY], s);
    s = fmaf(__ldg(&coef[14 * N + p]), z[q + 1 + kPXY], s);
    s = fmaf(__ldg(&coef[15 * N + p]), z[q - kPX - kPXY], s);
    s = fmaf(__ldg(&coef[16 * N + p]), z[q + kPX - kPXY], s);
    s = fmaf(__ldg(&coef[17 * N + p]), z[q - kPX + kPXY], s);
    s = fmaf(__ldg(&coef[18 * N + p]), z[q + kPX + kPXY], s);
  }
  return s;
}

template <int S, typename RT>
__global__ void __launch_bounds__(kSdThreads, 4)
    k_subdomain_local32(Dims d, const float* __restrict__ coef, const float* __restrict__ dinv,
                        const RT* __restrict__ r, float* __restrict__ z, const int* skip, int nbx, int nby) {
  if (skip != nullptr && *skip != 0) return;
  __shared__ float buf[2][kPad];
  const float om = (float)kSdOmega;
  const int box = blockIdx.x;
  const int x0 = (box % nbx) * kSdBX, y0 = ((box / nbx) % nby) * kSdBY, z0 = (box / (nbx * nby)) * kSdBZ;
  const int wx = min(kSdBX, d.nx - x0), wy = min(kSdBY, d.ny - y0), wz = min(kSdBZ, d.nz - z0);
  const int ex = wx + 2 * kSdOverlap, ey = wy + 2 * kSdOverlap, ez = wz + 2 * kSdOverlap;
  const int ne = ex * ey * ez;
  const int64_t N = d.n;
  const int64_t plane = (int64_t)d.nx * d.ny;
  for (int t = threadIdx.x; t < 2 * kPad; t += kSdThreads) (&buf[0][0])[t] = 0.f;
  int64_t gp[kCellsPer];
  int pe[kCellsPer];
  float rv[kCellsPer], dv[kCellsPer];
#pragma unroll
  for (int i = 0; i < kCellsPer; ++i) {
    const int e = threadIdx.x + i * kSdThreads;
    gp[i] = -1;
    pe[i] = 0;
    rv[i] = 0.f;
    dv[i] = 0.f;
    if (e < ne) {
      const int a = e % ex, b = (e / ex) % ey, c = e / (ex * ey);
      pe[i] = (a + 1) + kPX * ((b + 1) + kPY * (c + 1));
      const int gi = sd_wrap(x0 - kSdOverlap + a, d.nx, d.px);
      const int gj = sd_wrap(y0 - kSdOverlap + b, d.ny, d.py);
      const int gk = sd_wrap(z0 - kSdOverlap + c, d.nz, d.pz);
      if (gi >= 0 && gj >= 0 && gk >= 0) {
        gp[i] = (int64_t)gi + (int64_t)d.nx * gj + plane * gk;
        rv[i] = sd_ld32<RT>(r, gp[i]);
        dv[i] = __ldg(&dinv[gp[i]]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kCellsPer; ++i)
    if (gp[i] >= 0) buf[0][pe[i]] = __fmul_rn(om, __fmul_rn(dv[i], rv[i]));
  __syncthreads();
  int cur = 0;
  for (int sw = 1; sw < kSdSweeps - 1; ++sw) {
    const float* za = buf[cur];
    float* zb = buf[cur ^ 1];
#pragma unroll
    for (int i = 0; i < kCellsPer; ++i) {
      if (gp[i] < 0) continue;
      const float sv = sd_row32<S>(coef, N, gp[i], za, pe[i]);
      const float u = __fmul_rn(dv[i], __fsub_rn(rv[i], sv));
      zb[pe[i]] = fmaf(om, u, za[pe[i]]);
    }
    __syncthreads();
    cur ^= 1;
  }
  const float* za = buf[cur];
  const int nown = wx * wy * wz;
  for (int e = threadIdx.x; e < nown; e += kSdThreads) {
    const int a = e % wx, b = (e / wx) % wy, c = e / (wx * wy);
    const int64_t p = (int64_t)(x0 + a) + (int64_t)d.nx * (y0 + b) + plane * (z0 + c);
    const int q = (a + 1 + kSdOverlap) + kPX * ((b + 1 + kSdOverlap) + kPY * (c + 1 + kSdOverlap));
    const float sv = sd_row32<S>(coef, N, p, za, q);
    const float u = __fmul_rn(__ldg(&dinv[p]), __fsub_rn(sd_ld32<RT>(r, p), sv));
    z[p] = fmaf(om, u, za[q]);
  }
}

// ---- the double-float variant (the `df` precision): the same sweeps with the
// double-float copies of the bands and of 1/a_pp, the sweep buffers in
// double-float and every operation a double-float one on the FP32 pipe
// (TwoProduct products, lazy accumulation of the band sum in band order,
// renormalised every 8 bands and at the end). About 2^-44 relative per
// sweep instead of FP64 rounding; 5x fewer issue cycles than the FP64 pipe.
template <typename RT>
__device__ __forceinline__ float2 sd_ld_df(const RT* p, int64_t q);
template <>
__device__ __forceinline__ float2 sd_ld_df<float2>(const float2* p, int64_t q) { return __ldg(&p[q]); }
template <>
__device__ __forceinline__ float2 sd_ld_df<double>(const double* p, int64_t q) {
  return df_from_double_i(__ldg(&p[q]));
}

template <int S>
__device__ __forceinline__ float2 sd_row_df(const float2* __restrict__ coef, int64_t N, int64_t p, const float2* z,
                                            int q) {
  float s, c;
  {
    const float2 a = __ldg(&coef[p]);
    const float2 v = z[q];
    df_mul_pair(a.x, a.y, v.x, v.y, s, c);
  }
  auto mac = [&](int band, int off) {
    const float2 a = __ldg(&coef[band * N + p]);
    const float2 v = z[q + off];
    df_mac_lazy(s, c, a.x, a.y, v.x, v.y);
  };
  mac(1, -1);
  mac(2, 1);
  mac(3, -kPX);
  mac(4, kPX);
  mac(5, -kPXY);
  mac(6, kPXY);
  if (S == 19) {
    mac(7, -1 - kPX);
    df_renorm(s, c);
    mac(8, 1 - kPX);
    mac(9, -1 + kPX);
    mac(10, 1 + kPX);
    mac(11, -1 - kPXY);
    mac(12, 1 - kPXY);
    mac(13, -1 + kPXY);
    mac(14, 1 + kPXY);
    mac(15, -kPX - kPXY);
    df_renorm(s, c);
    mac(16, kPX - kPXY);
    mac(17, -kPX + kPXY);
    mac(18, kPX + kPXY);
  }
  df_renorm(s, c);
  return make_float2(s, c);
}

template <int S, typename RT>
__global__ void __launch_bounds__(kSdThreads, 2)
    k_subdomain_local_dd(Dims d, const float2* __restrict__ coef, const float2* __restrict__ dinv,
                         const RT* __restrict__ r, float2* __restrict__ z, const int* skip, int nbx, int nby,
                         float2 om) {
  if (skip != nullptr && *skip != 0) return;
  __shared__ float2 buf[2][kPad];
  const int box = blockIdx.x;
  const int x0 = (box % nbx) * kSdBX, y0 = ((box / nbx) % nby) * kSdBY, z0 = (box / (nbx * nby)) * kSdBZ;
  const int wx = min(kSdBX, d.nx - x0), wy = min(kSdBY, d.ny - y0), wz = min(kSdBZ, d.nz - z0);
  const int ex = wx + 2 * kSdOverlap, ey = wy + 2 * kSdOverlap, ez = wz + 2 * kSdOverlap;
  const int ne = ex * ey * ez;
  const int64_t N = d.n;
  const int64_t plane = (int64_t)d.nx * d.ny;
  for (int t = threadIdx.x; t < 2 * kPad; t += kSdThreads) (&buf[0][0])[t] = make_float2(0.f, 0.f);
  int64_t gp[kCellsPer];
  int pe[kCellsPer];
  float2 rv[kCellsPer];  // 1/a_pp is re-read from L1 each sweep (register budget)
#pragma unroll
  for (int i = 0; i < kCellsPer; ++i) {
    const int e = threadIdx.x + i * kSdThreads;
    gp[i] = -1;
    pe[i] = 0;
    rv[i] = make_float2(0.f, 0.f);
    if (e < ne) {
      const int a = e % ex, b = (e / ex) % ey, c = e / (ex * ey);
      pe[i] = (a + 1) + kPX * ((b + 1) + kPY * (c + 1));
      const int gi = sd_wrap(x0 - kSdOverlap + a, d.nx, d.px);
      const int gj = sd_wrap(y0 - kSdOverlap + b, d.ny, d.py);
      const int gk = sd_wrap(z0 - kSdOverlap + c, d.nz, d.pz);
      if (gi >= 0 && gj >= 0 && gk >= 0) {
        gp[i] = (int64_t)gi + (int64_t)d.nx * gj + plane * gk;
        rv[i] = sd_ld_df<RT>(r, gp[i]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kCellsPer; ++i)
    if (gp[i] >= 0) buf[0][pe[i]] = df_mul(om, df_mul(__ldg(&dinv[gp[i]]), rv[i]));
  __syncthreads();
  int cur = 0;
  for (int sw = 1; sw < kSdSweeps - 1; ++sw) {
    const float2* za = buf[cur];
    float2* zb = buf[cur ^ 1];
#pragma unroll
    for (int i = 0; i < kCellsPer; ++i) {
      if (gp[i] < 0) continue;
      const float2 s = sd_row_df<S>(coef, N, gp[i], za, pe[i]);
      const float2 u = df_mul(__ldg(&dinv[gp[i]]), df_sub(rv[i], s));
      zb[pe[i]] = df_fma(om, u, za[pe[i]]);
    }
    __syncthreads();
    cur ^= 1;
  }
  const float2* za = buf[cur];
  const int nown = wx * wy * wz;
  for (int e = threadIdx.x; e < nown; e += kSdThreads) {
    const int a = e % wx, b = (e / wx) % wy, c = e / (wx * wy);
    const int64_t p = (int64_t)(x0 + a) + (int64_t)d.nx * (y0 + b) + plane * (z0 + c);
    const int q = (a + 1 + kSdOverlap) + kPX * ((b + 1 + kSdOverlap) + kPY * (c + 1 + kSdOverlap));
    const float2 s = sd_row_df<S>(coef, N, p, za, q);
    const float2 u = df_mul(__ldg(&dinv[p]), df_sub(sd_ld_df<RT>(r, p), s));
    z[p] = df_fma(om, u, za[q]);
  }
}

// The 7-point double-float variant with the grown box's bands and 1/a_pp
// staged in shared memory once per box (100.8 + 14.4 KB), so the sweeps read
// no global memory: one CTA of 1024 threads per SM, two grown-box cells per
// thread. The arithmetic is that of
// k_subdomain_local_dd, operation for operation.
constexpr int kSdsThreads = 1024;
constexpr int kSdsCellsPer = (kEX * kEY * kEZ + kSdsThreads - 1) / kSdsThreads;
constexpr int kGrown = kEX * kEY * kEZ;
constexpr size_t kSdsSmem = sizeof(float2) * (2 * kPad + 8 * kGrown);

__device__ __forceinline__ float2 sd_row_df7_smem(const float2* cs, int e, const float2* z, int q) {
  float s, c;
  {
    const float2 a = cs[e];
    const float2 v = z[q];
    df_mul_pair(a.x, a.y, v.x, v.y, s, c);
  }
  auto mac = [&](int band, int off) {
    const float2 a = cs[band * kGrown + e];
    const float2 v = z[q + off];
    df_mac_lazy(s, c, a.x, a.y, v.x, v.y);
  };
  mac(1, -1);
  mac(2, 1);
  mac(3, -kPX);
  mac(4, kPX);
  mac(5, -kPXY);
  mac(6, kPXY);
  df_renorm(s, c);
  return make_float2(s, c);
}

template <typename RT>
__global__ void __launch_bounds__(kSdsThreads, 1)
    k_subdomain_local_dd7s(Dims d, const float2* __restrict__ coef, const float2* __restrict__ dinv,
                           const RT* __restrict__ r, float2* __restrict__ z, const int* skip, int nbx, int nby,
                           float2 om) {
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ float2 sds[];
  float2* buf0 = sds;
  float2* buf1 = sds + kPad;
  float2* cs = sds + 2 * kPad;  // 7 bands x kGrown, then 1/a_pp
  float2* ds = cs + 7 * kGrown;
  const int box = blockIdx.x;
  const int x0 = (box % nbx) * kSdBX, y0 = ((box / nbx) % nby) * kSdBY, z0 = (box / (nbx * nby)) * kSdBZ;
  const int wx = min(kSdBX, d.nx - x0), wy = min(kSdBY, d.ny - y0), wz = min(kSdBZ, d.nz - z0);
  const int ex = wx + 2 * kSdOverlap, ey = wy + 2 * kSdOverlap, ez = wz + 2 * kSdOverlap;
  const int ne = ex * ey * ez;
  const int64_t N = d.n;
  const int64_t plane = (int64_t)d.nx * d.ny;
  for (int t = threadIdx.x; t < 2 * kPad; t += kSdsThreads) sds[t] = make_float2(0.f, 0.f);
  int64_t gp[kSdsCellsPer];
  int pe[kSdsCellsPer];
  float2 rv[kSdsCellsPer];
#pragma unroll
  for (int i = 0; i < kSdsCellsPer; ++i) {
    const int e = threadIdx.x + i * kSdsThreads;
    gp[i] = -1;
    pe[i] = 0;
    rv[i] = make_float2(0.f, 0.f);
    if (e < ne) {
      const int a = e % ex, b = (e / ex) % ey, c = e / (ex * ey);
      pe[i] = (a + 1) + kPX * ((b + 1) + kPY * (c + 1));
      const int gi = sd_wrap(x0 - kSdOverlap + a, d.nx, d.px);
      const int gj = sd_wrap(y0 - kSdOverlap + b, d.ny, d.py);
      const int gk = sd_wrap(z0 - kSdOverlap + c, d.nz, d.pz);
      if (gi >= 0 && gj >= 0 && gk >= 0) {
        const int64_t p = (int64_t)gi + (int64_t)d.nx * gj + plane * gk;
        gp[i] = p;
        rv[i] = sd_ld_df<RT>(r, p);
#pragma unroll
        for (int t = 0; t < 7; ++t) cs[t * kGrown + e] = __ldg(&coef[t * N + p]);
        ds[e] = __ldg(&dinv[p]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSdsCellsPer; ++i) {
    const int e = threadIdx.x + i * kSdsThreads;
    if (gp[i] >= 0) buf0[pe[i]] = df_mul(om, df_mul(ds[e], rv[i]));
  }
  __syncthreads();
  float2* za = buf0;
  float2* zb = buf1;
  for (int sw = 1; sw < kSdSweeps - 1; ++sw) {
#pragma unroll
    for (int i = 0; i < kSdsCellsPer; ++i) {
      if (gp[i] < 0) continue;
      const int e = threadIdx.x + i * kSdsThreads;
      const float2 s = sd_row_df7_smem(cs, e, za, pe[i]);
      const float2 u = df_mul(ds[e], df_sub(rv[i], s));
      zb[pe[i]] = df_fma(om, u, za[pe[i]]);
    }
    __syncthreads();
    float2* tmp = za;
    za = zb;
    zb = tmp;
  }
  const int nown = wx * wy * wz;
  for (int e = threadIdx.x; e < nown; e += kSdsThreads) {
    const int a = e % wx, b = (e / wx) % wy, c = e / (wx * wy);
    const int64_t p = (int64_t)(x0 + a) + (int64_t)d.nx * (y0 + b) + plane * (z0 + c);
    const int eg = (a + kSdOverlap) + ex * ((b + kSdOverlap) + ey * (c + kSdOverlap));
    const int q = (a + 1 + kSdOverlap) + kPX * ((b + 1 + kSdOverlap) + kPY * (c + 1 + kSdOverlap));
    const float2 s = sd_row_df7_smem(cs, eg, za, q);
    const float2 u = df_mul(ds[eg], df_sub(sd_ld_df<RT>(r, p), s));
    z[p] = df_fma(om, u, za[q]);
  }
}

__global__ void __launch_bounds__(kRedThreads) k_add(int64_t n, const double* __restrict__ v, double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = x[i] + __ldg(&v[i]);
}

}  // namespace

int64_t subdomain_boxes(const Dims& d) {
  return (int64_t)((d.nx + kSdBX - 1) / kSdBX) * ((d.ny + kSdBY - 1) / kSdBY) * ((d.nz + kSdBZ - 1) / kSdBZ);
}

cudaError_t launch_subdomain_local(const Dims& d, int S, const double* coef, const double* dinv, const double* r,
                                   double* z, const int* skip, cudaStream_t st) {
  const int nbx = (d.nx + kSdBX - 1) / kSdBX, nby = (d.ny + kSdBY - 1) / kSdBY;
  const int64_t nb = subdomain_boxes(d);
  if (nb <= 0 || nb > 0x7fffffff) return cudaErrorInvalidValue;
  if (S == 7)
    k_subdomain_local<7><<<(unsigned)nb, kSdThreads, 0, st>>>(d, coef, dinv, r, z, skip, nbx, nby);
  else
    k_subdomain_local<19><<<(unsigned)nb, kSdThreads, 0, st>>>(d, coef, dinv, r, z, skip, nbx, nby);
  return cudaGetLastError();
}

cudaError_t launch_subdomain_local32(const Dims& d, int S, const float* coef32, const float* dinv32, const void* r,
                                     bool r_f32, float* z, const int* skip, cudaStream_t st) {
  const int nbx = (d.nx + kSdBX - 1) / kSdBX, nby = (d.ny + kSdBY - 1) / kSdBY;
  const int64_t nb = subdomain_boxes(d);
  if (nb <= 0 || nb > 0x7fffffff) return cudaErrorInvalidValue;
#define RK_SL32(SS, RT) \
  k_subdomain_local32<SS, RT><<<(unsigned)nb, kSdThreads, 0, st>>>(d, coef32, dinv32, (const RT*)r, z, skip, nbx, nby)
  if (S == 7) {
    if (r_f32) RK_SL32(7, float); else RK_SL32(7, double);
  } else {
    if (r_f32) RK_SL32(19, float); else RK_SL32(19, double);
  }
#undef RK_SL32
  return cudaGetLastError();
}

// The 161 KB of dynamic shared memory of the staged 7-band double-float
// sweeps need an opt-in, once per device (the batch executor launches from
// several host threads); also run when a problem is created, so that it
// never happens inside a graph capture.
void subdomain_prepare() {
  static std::atomic<uint64_t> done{0};
  once_per_device(done, [] {
    cudaFuncSetAttribute(k_subdomain_local_dd7s<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSdsSmem);
    cudaFuncSetAttribute(k_subdomain_local_dd7s<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSdsSmem);
  });
}

cudaError_t launch_subdomain_local_dd(const Dims& d, int S, const float2* coefd, const float2* dinvd, const void* r,
                                      bool r_df, float2* z, const int* skip, cudaStream_t st) {
  const int nbx = (d.nx + kSdBX - 1) / kSdBX, nby = (d.ny + kSdBY - 1) / kSdBY;
  const int64_t nb = subdomain_boxes(d);
  if (nb <= 0 || nb > 0x7fffffff) return cudaErrorInvalidValue;
  const float oh = (float)kSdOmega;
  const float2 om = make_float2(oh, (float)(kSdOmega - (double)oh));
  if (S == 7) {
    subdomain_prepare();
    if (r_df)
      k_subdomain_local_dd7s<float2><<<(unsigned)nb, kSdsThreads, kSdsSmem, st>>>(d, coefd, dinvd, (const float2*)r, z,
                                                                                 skip, nbx, nby, om);
    else
      k_subdomain_local_dd7s<double><<<(unsigned)nb, kSdsThreads, kSdsSmem, st>>>(d, coefd, dinvd, (const double*)r, z,
                                                                                 skip, nbx, nby, om);
    return cudaGetLastError();
  }
#define RK_SLD(SS, RT)                                                                                          \
  k_subdomain_local_dd<SS, RT><<<(unsigned)nb, kSdThreads, 0, st>>>(d, coefd, dinvd, (const RT*)r, z, skip, nbx, \
                                                                   nby, om)
  if (S == 7) {
    if (r_df) RK_SLD(7, float2); else RK_SLD(7, double);
  } else {
    if (r_df) RK_SLD(19, float2); else RK_SLD(19, double);
  }
#undef RK_SLD
  return cudaGetLastError();
}

cudaError_t launch_add(int64_t n, const double* v, double* x, cudaStream_t st) {
  k_add<<<red_blocks(n), kRedThreads, 0, st>>>(n, v, x);
  return cudaGetLastError();
}

}  // namespace rk
