// Row-tiled double-float X P on the tensor cores (the in-place recycle
// updates C <- W_hat QC and U <- W PU of Algorithm 3).
//
// A double-float product cannot run on BF16 tensor cores directly, but an
// integer one can, exactly: each row r of X = [A, diag(bscale) Bm] is scaled
// by a power of two 2^-E_r (|x| < 2^E_r over the row) and written as seven
// signed digits, x = 2^E_r sum_i s_i 256^-i + (below 2^(E_r - 57)), with
// |s_1|, |s_7| <= 256, |s_4| <= 192 and the others <= 128; each column c of
// P likewise with 2^F_c and digits t_j (|t_1| <= 256, the others <= 128).
// BF16 holds such integers exactly (at most 8 significant bits), a digit
// product is an integer of at most 2^16, and FP32 accumulation is exact
// while a sum stays below 2^24. The products are grouped by level L = i + j:
//   X P = 2^(E_r + F_c) sum_L 256^-L (sum_{i+j=L} s_i t_j),
// each level accumulated exactly in its own 32 TMEM columns (with K <= 64
// every level sum stays below 2^23.6). Levels 2..8 are kept (28 digit pairs); what
// is dropped lies below 2^-50 of |X||P|, and seven digits hold all 48 bits
// of a double-float value within 2^8 of its row's largest. For digit row i,
// one MMA with B = [t_1 | ... | t_(8-i)] (N = 32 (8 - i)) accumulates every
// level i + j at once into TMEM columns 32 (i - 1) .. 223, so a 16-wide K
// step is 7 MMAs. The epilogue reads the 7 level sums, combines them in
// double-float (every term exact) and applies 2^(E_r + F_c).
//
// One block per SM, a persistent loop over tiles of 128 rows (one TMEM lane
// per row). A loader warp brings each tile of X (and the row scales) into
// shared memory by bulk asynchronous copies, two tiles ahead (three tile
// buffers). Eight producer warps: warp w owns rows 32 (w % 4) .. +31 (its
// TMEM lanes) and half w / 4 of K. Per tile a producer finds its half-row
// maximum, trades it with the warp owning the other half (a 64-thread named
// barrier), writes per 16 columns of K its 8 x 7 digits into one of two
// digit buffers in TMEM (the MMAs' A operand) and arrives on the buffer's
// "full" barrier; the MMA issuer warp waits for all eight, issues the 7 MMAs
// (B, the digits of P, in shared memory) and commits them to the buffer's
// "free" barrier. After the tile's last MMAs a commit on "tmem full"
// releases the epilogue, in which each producer reads its lanes' level sums
// for its output columns; "tmem free" lets the issuer start the next tile.
// No block-wide barrier inside the loop. The digits of P are made once per
// launch by k_tc_digits_p.
#include <cuda_bf16.h>

#include "rk_internal.h"
#include "rk_df.cuh"
#include "rk_tcgen05.cuh"

namespace rk {

namespace {

constexpr int kTcRows = 128;                    // rows per tile = MMA M = TMEM lanes
constexpr int kTcProducers = 8;                 // producer warps (two per row: K halves)
constexpr int kTcThreads = 32 * (kTcProducers + 2);  // + the MMA issuer and the loader warps
constexpr int kTcDigits = 7;                    // digits per operand
constexpr int kTcCols = 32;                     // output columns per level (MMA N per digit of P)
constexpr int kTcTmem = 512;                    // 7 levels x 32 accumulator columns, then the A digits
constexpr int kTcADig = 256;                    // TMEM column of the first A digit buffer
constexpr int kTcKMax = 64;                     // K <= 64 keeps every level sum exact
constexpr int kTcADigCols = 64;                 // TMEM columns per A digit buffer (7 planes x 8 used)
constexpr int kTcXStages = 3;                   // X tiles in shared memory (two prefetched ahead)
constexpr int kTcBRows = kTcDigits * kTcCols;   // 224 rows of B: (digit j, column c)
constexpr int kTcBBytes = kTcBRows * kTcKMax * 2;             // 28 KB
constexpr int kTcXBuf = kTcRows * kTcKMax * (int)sizeof(float2);  // 64 KB per X tile
constexpr size_t kTcSmem = kTcXStages * (size_t)kTcXBuf + kTcBBytes + kTcXStages * kTcRows * sizeof(double);

// element offset of (row, k) in a K-major canonical operand with kg 8-wide
// core-matrix columns along K
__host__ __device__ __forceinline__ int tc_off(int row, int k, int kg) {
  return (((row >> 3) * kg + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

// Digits of P (np x nc, FP64, column-major, leading dimension np): B rows
// n = 32 j + c hold digit j+1 of column c over k = 0..kp-1 (zero outside
// np x nc); fexp[c] = F_c. Seven base-256 digits hold all 53 bits.
__global__ void k_tc_digits_p(int np, int nc, int kp, const double* __restrict__ P, __nv_bfloat16* __restrict__ B,
                              int* __restrict__ fexp) {
  __shared__ int fs[kTcCols];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int c = warp; c < kTcCols; c += nwarp) {
    double m = 0.0;
    if (c < nc)
      for (int q = lane; q < np; q += 32) m = fmax(m, fabs(P[(int64_t)c * np + q]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) fs[c] = m > 0.0 ? ilogb(m) + 1 : 0;  // |P_qc| < 2^F_c
  }
  __syncthreads();
  const int kg = kp >> 3;
  for (int t = threadIdx.x; t < kTcCols * kp; t += blockDim.x) {
    const int c = t / kp, q = t - c * kp;
    double y = (c < nc && q < np) ? ldexp(P[(int64_t)c * np + q], -fs[c]) : 0.0;
    for (int j = 0; j < kTcDigits; ++j) {
      y *= 256.0;
      const double d = rint(y);
      y -= d;
      B[tc_off(j * kTcCols + c, q, kg)] = __double2bfloat16(d);
    }
  }
  if (threadIdx.x < kTcCols) fexp[threadIdx.x] = fs[threadIdx.x];
}

// Two digits (integers of at most 9 significant bits, so the low 16 bits of
// their FP32 encodings are zero) as a BF16 pair: the high halves, lo first.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// x * 2^ex for the epilogue: exponent arithmetic when x and the result are
// normal numbers, ldexpf otherwise
__device__ __forceinline__ float scale_pow2(float x, int ex) {
  const unsigned u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xffu);
  if (e >= 1 && e <= 254 && e + ex >= 1 && e + ex <= 254) return __uint_as_float(u + ((unsigned)ex << 23));
  return ldexpf(x, ex);
}

// ---- FP64 operands (the RK_FP64 / RK_MIXED basis). A row's values are cut
// against 2^E (|x| < 2^E over the row) into the signed fixed-point integer
// F = trunc(x 2^(56 - E)) (|F| < 2^56: every bit of x within 2^3 of the
// row's largest, the rest truncated below 2^(E - 56)), taken from the
// IEEE-754 bits with integer operations, and F into seven balanced base-256
// digits by rounding shifts from the top: d_1 = round(F / 2^48) (|d_1| <=
// 256), each next digit the rounded remainder (|d_i| <= 128), so
// F = sum_i d_i 2^(56 - 8i) exactly. The level sums S_L (exact integers
// below 2^24 in FP32) are combined exactly in 64-bit integers
// (hi = S_2 2^24 + S_3 2^16 + S_4 2^8 + S_5, lo = S_6 2^16 + S_7 2^8 + S_8)
// and rounded once, fma(hi, 2^24, lo), in FP64.

// the biased exponent field of x (0 for zeros and subnormals, which count as 0)
__device__ __forceinline__ int f64_expbits(double x) {
  return (int)((unsigned)(__double_as_longlong(x) >> 52) & 0x7ffu);
}

// F = trunc(x 2^(56 - E)) with E = emax - 1022 (emax the row's largest
// exponent field), from the bits of x
__device__ __forceinline__ long long f64_fixed56(double x, int emax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)((b >> 52) & 0x7ffu);
  if (eb == 0) return 0;
  const unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;
  const int sh = eb - emax + 3;  // <= 3
  unsigned long long f;
  if (sh >= 0)
    f = m << sh;
  else
    f = sh > -60 ? (m >> (-sh)) : 0ull;
  return (b >> 63) ? -(long long)f : (long long)f;
}

// exact FP32 integer value (|v| < 2^25) to int, from the bits
__device__ __forceinline__ int f32_int_exact(float v) {
  const unsigned u = __float_as_uint(v);
  const int e = (int)((u >> 23) & 0xffu);
  if (e < 127) return 0;  // |v| < 1: 0 (level sums are integers)
  const int m = (int)((u & 0x7fffffu) | 0x800000u);
  const int r = e >= 150 ? (m << (e - 150)) : (m >> (150 - e));
  return (u >> 31) ? -r : r;
}

// exact int64 (|v| < 2^53) to FP64, from the bits
__device__ __forceinline__ double i64_to_f64_exact(long long v) {
  if (v == 0) return 0.0;
  const unsigned long long neg = v < 0 ? 1ull : 0ull;
  unsigned long long a = neg ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll((long long)a);   // a < 2^53: lz >= 11
  const int e = 63 - lz;                  // a in [2^e, 2^(e+1))
  a <<= (52 - e);                         // 53 significant bits, leading bit at 52
  const unsigned long long bits = (neg << 63) | ((unsigned long long)(e + 1023) << 52) | (a & 0xfffffffffffffull);
  return __longlong_as_double((long long)bits);
}

template <bool F64>
__global__ void __launch_bounds__(kTcThreads, 1) k_dfgemm_tc(DFGemmArgs a, const __nv_bfloat16* __restrict__ bdig,
                                                                const int* __restrict__ fexp, int kp, int bulk_ok,
                                                                int* err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  float2* xs = reinterpret_cast<float2*>(tsm);                     // [kTcXStages][kTcKMax][kTcRows] X tiles
  unsigned char* sB = tsm + kTcXStages * kTcXBuf;                   // digits of P
  double* bsv = reinterpret_cast<double*>(sB + kTcBBytes);          // [kTcXStages][kTcRows] row scales
  __shared__ __align__(8) uint64_t xfull[kTcXStages], xfree[kTcXStages], dfull[2], dfree[2], tfull, tfree;
  __shared__ uint32_t tslot;
  __shared__ int fs[kTcCols];
  __shared__ float rmax[2][2][kTcRows];  // [tile parity][K half][row]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = a.na + a.nb;
  const int kg = kp >> 3, nks = kp >> 4;
  {
    const uint4* src = reinterpret_cast<const uint4*>(bdig);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    const int n16 = kTcBRows * kp * 2 / 16;
    for (int i = tid; i < n16; i += kTcThreads) dst[i] = __ldg(&src[i]);
  }
  if (tid < kTcCols) fs[tid] = fexp[tid];
  if (warp == 0) tc_alloc(&tslot, kTcTmem);
  if (tid == 0) {
    for (int b = 0; b < kTcXStages; ++b) {
      mbar_init(&xfull[b], 1);
      mbar_init(&xfree[b], kTcProducers);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&dfull[b], kTcProducers);
      mbar_init(&dfree[b], 1);
    }
    mbar_init(&tfull, 1);
    mbar_init(&tfree, kTcProducers);
    mbar_init_fence();
  }
  fence_async_shared();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t taddr = tslot;
  const int64_t ntiles = (a.n + kTcRows - 1) / kTcRows;
  // a tile comes by bulk copies when it is full and the operands are aligned
  // (only the ragged last tile, or every tile of unaligned operands, does not)
  auto is_bulk = [&](int64_t t) { return bulk_ok != 0 && (t + 1) * kTcRows <= a.n; };
  bool ok = true;
  auto wait = [&](uint64_t* bar, unsigned parity) { ok = mbar_wait_bounded(bar, parity) && ok; };
  if (warp == kTcProducers + 1) {
    // ---------------------------------------------------------------- loader
    if (lane == 0) {
      auto issue = [&](int64_t t, int b) {
        const int64_t r0 = t * kTcRows;
        const unsigned bytes = kTcRows * (unsigned)sizeof(float2);
        fence_async_shared();
        mbar_arrive_expect_tx(&xfull[b], bytes * np + (a.bscale ? kTcRows * (unsigned)sizeof(double) : 0u));
        for (int q = 0; q < np; ++q) {
          const float2* src = q < a.na ? a.A + (int64_t)q * a.lda + r0 : a.Bm + (int64_t)(q - a.na) * a.ldb + r0;
          bulk_g2s(xs + ((int64_t)b * kTcKMax + q) * kTcRows, src, bytes, &xfull[b]);
        }
        if (a.bscale) bulk_g2s(bsv + b * kTcRows, a.bscale + r0, kTcRows * (unsigned)sizeof(double), &xfull[b]);
      };
      // the first two tiles, then one tile per producer tile finished: tile
      // it + 2 goes into the buffer tile it - 1 has released
      for (int p = 0; p < 2; ++p) {
        const int64_t t = blockIdx.x + (int64_t)p * gridDim.x;
        if (t < ntiles && is_bulk(t)) issue(t, p);
      }
      int it = 0;
      for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int64_t nx = tile + 2 * (int64_t)gridDim.x;
        if (nx < ntiles && is_bulk(nx)) {
          const int nb = (it + 2) % kTcXStages;
          if (it >= 1) wait(&xfree[nb], (unsigned)(((it - 1) / kTcXStages) & 1));
          issue(nx, nb);
        }
      }
    }
  } else if (warp == kTcProducers) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t bdesc0 = smem_u32(sB);
      int cc = 0, it = 0;
      for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        if (it >= 1) wait(&tfree, (unsigned)((it - 1) & 1));  // the previous epilogue has read TMEM
        for (int ks = 0; ks < nks; ++ks, ++cc) {
          const int b = cc & 1;
          wait(&dfull[b], (unsigned)((cc >> 1) & 1));
          tc_fence_after_sync();
#pragma unroll
          for (int i = 0; i < kTcDigits; ++i) {
            const uint64_t bd = tc_smem_desc(bdesc0 + ks * 256, 128, kg * 128);
            tc_mma_bf16_ta(taddr + kTcCols * i, taddr + kTcADig + b * kTcADigCols + 8 * i, bd,
                           tc_idesc_bf16(kTcRows, kTcCols * (kTcDigits - i)), (ks > 0 || i > 0) ? 1u : 0u);
          }
          tc_commit(&dfree[b]);
        }
        tc_commit(&tfull);
      }
    }
  } else {
    // ---------------------------------------------------------------- producers
    const int rl = 32 * (warp & 3) + lane;  // row in the tile = TMEM lane
    const int half = warp >> 2;             // K half for digits, column half in the epilogue
    const int pairbar = 1 + (warp & 3);     // named barrier of warps w and w + 4
    int cc = 0, it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int xb = it % kTcXStages;
      const int64_t r0 = tile * kTcRows;
      const int64_t row = r0 + rl;
      const bool valid = row < a.n;
      float2* X = xs + (int64_t)xb * kTcKMax * kTcRows;
      double* bs = bsv + xb * kTcRows;
      if (is_bulk(tile)) {
        wait(&xfull[xb], (unsigned)((it / kTcXStages) & 1));
      } else {
        // this thread's own elements (its row, its K half) and row scale
        for (int ks = 0; ks < nks; ++ks)
          for (int e = 0; e < 8; ++e) {
            const int q = ks * 16 + half * 8 + e;
            if (q >= np) break;
            float2 v = make_float2(0.f, 0.f);
            if (valid)
              v = q < a.na ? __ldg(&a.A[(int64_t)q * a.lda + row]) : __ldg(&a.Bm[(int64_t)(q - a.na) * a.ldb + row]);
            X[q * kTcRows + rl] = v;
          }
        if (a.bscale) bs[rl] = valid ? __ldg(&a.bscale[row]) : 0.0;
      }
      float2 sc = make_float2(1.f, 0.f);
      float scale = 1.f;
      int E = 0, emax = 0;
      double* Xd = reinterpret_cast<double*>(X);
      if constexpr (F64) {
        // the B columns scaled in place (one FP64 product each), then the
        // largest exponent field of the half-row, traded with the partner warp
        const double scd = a.bscale ? bs[rl] : 1.0;
        int em = 0;
        for (int ks = 0; ks < nks; ++ks)
          for (int e = 0; e < 8; ++e) {
            const int q = ks * 16 + half * 8 + e;
            if (q >= np) break;
            double x = Xd[q * kTcRows + rl];
            if (q >= a.na && a.bscale) {
              x *= scd;
              Xd[q * kTcRows + rl] = x;
            }
            em = max(em, f64_expbits(x));
          }
        rmax[it & 1][half][rl] = __int_as_float(em);
        named_barrier_sync(pairbar, 64);
        emax = max(__float_as_int(rmax[it & 1][0][rl]), __float_as_int(rmax[it & 1][1][rl]));
        E = emax > 0 ? emax - 1022 : 0;  // |x| < 2^E over the row
      } else {
        sc = a.bscale ? df_from_double_i(bs[rl]) : make_float2(1.f, 0.f);
        // half-row maximum of the high words; for the B part max |b| |s| with
        // 2^-20 of headroom, which bounds the double-float products taken
        // with the digits (their high words differ from b_hi s_hi by < 2^-22)
        float mxa = 0.f, mxb = 0.f;
        for (int ks = 0; ks < nks; ++ks)
          for (int e = 0; e < 8; ++e) {
            const int q = ks * 16 + half * 8 + e;
            if (q >= np) break;
            const float xh = fabsf(X[q * kTcRows + rl].x);
            if (q < a.na)
              mxa = fmaxf(mxa, xh);
            else
              mxb = fmaxf(mxb, xh);
          }
        float mx = fmaxf(mxa, mxb * fabsf(sc.x) * 1.00000095367431640625f);
        rmax[it & 1][half][rl] = mx;
        named_barrier_sync(pairbar, 64);
        mx = fmaxf(rmax[it & 1][0][rl], rmax[it & 1][1][rl]);
        E = mx > 0.f ? ilogbf(mx) + 1 : 0;
        E = E < -125 ? -125 : (E > 126 ? 126 : E);  // keep 2^-E a normal FP32 number
        scale = __int_as_float((127 - E) << 23);
      }
      for (int ks = 0; ks < nks; ++ks, ++cc) {
        const int b = cc & 1;
        if (cc >= 2) wait(&dfree[b], (unsigned)(((cc >> 1) - 1) & 1));  // the MMAs that read it last
        // this warp's lanes, this K half's 4 columns of each digit plane
        const uint32_t ta = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + kTcADig + b * kTcADigCols + 4 * half;
        if constexpr (F64) {
          // the 8 elements of this thread's row and K half: fixed-point
          // integers, then balanced base-256 digits top down
          long long rem[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int q = ks * 16 + half * 8 + e;
            rem[e] = q < np ? f64_fixed56(Xd[q * kTcRows + rl], emax) : 0ll;
          }
#pragma unroll
          for (int i = 0; i < kTcDigits; ++i) {
            const int sh = 48 - 8 * i;
            float d[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              long long t = rem[e];
              if (i < kTcDigits - 1) {
                t = (rem[e] + (1ll << (sh - 1))) >> sh;  // rounded (arithmetic shift)
                rem[e] -= t << sh;
              }
              d[e] = (float)(int)t;  // |t| <= 256: exact
            }
            tc_store4(ta + 8 * i, pack_bf16(d[0], d[1]), pack_bf16(d[2], d[3]), pack_bf16(d[4], d[5]),
                      pack_bf16(d[6], d[7]));
          }
        } else {
        // The 8 elements of this thread's row and K half, digit by digit
        // (ILP 8). Digit i is yh rounded to a multiple of 256^-i, taken as
        // (yh + 1.5 2^(23-8i)) - 1.5 2^(23-8i) (the sum's ulp is 256^-i),
        // subtracted exactly and scaled by 256^i. The low word joins the
        // remainder after digit 3 (Fast2Sum: the remainder is a multiple of
        // ulp(yh) >= 2 |yl| or zero) and its rounding error before digit 7.
        float yh[8], yl[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int q = ks * 16 + half * 8 + e;
          float2 x = q < np ? X[q * kTcRows + rl] : make_float2(0.f, 0.f);
          if (q >= a.na && q < np) x = df_mul(x, sc);
          yh[e] = __fmul_rn(x.x, scale);  // exact (power of two)
          yl[e] = __fmul_rn(x.y, scale);
        }
        auto digit = [&](int i, bool keep_rest) {
          const float sig = __int_as_float((127 + 23 - 8 * (i + 1)) << 23) * 1.5f;
          const float up = __int_as_float((127 + 8 * (i + 1)) << 23);
          float d[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float sv = __fsub_rn(__fadd_rn(yh[e], sig), sig);
            if (keep_rest) yh[e] = __fsub_rn(yh[e], sv);
            d[e] = __fmul_rn(sv, up);
          }
          tc_store4(ta + 8 * i, pack_bf16(d[0], d[1]), pack_bf16(d[2], d[3]), pack_bf16(d[4], d[5]),
                    pack_bf16(d[6], d[7]));
        };
        digit(0, true);
        digit(1, true);
        digit(2, true);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float t = __fadd_rn(yh[e], yl[e]);
          yl[e] = __fsub_rn(yl[e], __fsub_rn(t, yh[e]));
          yh[e] = t;
        }
        digit(3, true);
        digit(4, true);
        digit(5, true);
#pragma unroll
        for (int e = 0; e < 8; ++e) yh[e] = __fadd_rn(yh[e], yl[e]);
        digit(6, false);
        }
        tc_wait_store();
        tc_fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&dfull[b]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&xfree[xb]);  // done with this X tile
      // epilogue: this warp's 32 lanes, output columns 16 half .. +15
      wait(&tfull, (unsigned)(it & 1));
      tc_fence_after_sync();
      // groups of 8 of this warp's 16 output columns that exist
      for (int g = 0; g < 2 && 16 * half + 8 * g < a.nc; ++g) {
        const int c0 = 16 * half + 8 * g;
        const uint32_t tl = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + c0;
        float sh[8], sl[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) sh[u] = sl[u] = 0.f;
        uint32_t lv[kTcDigits][8];
#pragma unroll
        for (int L = 2; L <= kTcDigits + 1; ++L) tc_load8_async(tl + kTcCols * (L - 2), lv[L - 2]);
        tc_wait_load();
#pragma unroll
        for (int L = kTcDigits + 1; L >= 2 && !F64; --L) {
          const float w = __int_as_float((127 - 8 * L) << 23);  // 256^-L
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float p = __uint_as_float(lv[L - 2][u]) * w;  // exact
            const float s2 = sh[u] + p;
            const float bb = s2 - sh[u];
            sl[u] += (sh[u] - (s2 - bb)) + (p - bb);
            sh[u] = s2;
          }
        }
        if constexpr (F64) {
          if (valid) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int c = c0 + u;
              if (c < a.nc) {
                // sum_L S_L 256^(8-L) exactly in 64-bit integers, one rounding
                long long hi = 0, lo = 0;
#pragma unroll
                for (int L = 2; L <= 5; ++L) hi = (hi << 8) + f32_int_exact(__uint_as_float(lv[L - 2][u]));
#pragma unroll
                for (int L = 6; L <= kTcDigits + 1; ++L) lo = (lo << 8) + f32_int_exact(__uint_as_float(lv[L - 2][u]));
                const double v = fma(i64_to_f64_exact(hi), 16777216.0, i64_to_f64_exact(lo));
                reinterpret_cast<double*>(a.out)[(int64_t)c * a.ldo + row] = ldexp(v, E + fs[c] - 64);
              }
            }
          }
        } else if (valid) {
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int c = c0 + u;
            if (c < a.nc) {
              const float hi = sh[u] + sl[u];
              const float lo = sl[u] - (hi - sh[u]);
              const int ex = E + fs[c];
              reinterpret_cast<float2*>(a.out)[(int64_t)c * a.ldo + row] =
                  make_float2(scale_pow2(hi, ex), scale_pow2(lo, ex));
            }
          }
        }
      }
      tc_fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tfree);
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if (warp == 0) tc_dealloc(taddr, kTcTmem);
  if (!ok && err != nullptr) atomicExch(err, 3);
}

}  // namespace

size_t dfgemm_tc_ws_bytes() { return (size_t)kTcBBytes + kTcCols * sizeof(int); }

bool dfgemm_tc_supported(const DFGemmArgs& a, bool out_df) {
  const int np = a.na + a.nb;
  return out_df && a.accum == 0 && a.nc >= 2 && a.nc <= kTcCols && np >= 1 && np <= kTcKMax;
}

bool gemm_tc_f64_supported(int np, int nc, int accum) {
  return accum == 0 && nc >= 2 && nc <= kTcCols && np >= 1 && np <= kTcKMax;
}

void dfgemm_tc_prepare() {
  static std::atomic<uint64_t> done{0};
  once_per_device(done, [] {
    cudaFuncSetAttribute(k_dfgemm_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    cudaFuncSetAttribute(k_dfgemm_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  });
}

cudaError_t launch_dfgemm_tc(const DFGemmArgs& a, void* ws, int* err, cudaStream_t st, bool f64) {
  const int np = a.na + a.nb;
  const int kp = (np + 15) & ~15;
  __nv_bfloat16* bdig = reinterpret_cast<__nv_bfloat16*>(ws);
  int* fexp = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(ws) + kTcBBytes);
  k_tc_digits_p<<<1, 256, 0, st>>>(np, a.nc, kp, a.P, bdig, fexp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dfgemm_tc_prepare();
  const int64_t ntiles = (a.n + kTcRows - 1) / kTcRows;
  const int blocks = (int)(ntiles < kNumSM ? ntiles : kNumSM);
  if (blocks == 0) return cudaSuccess;
  // bulk copies need 16-byte aligned column segments
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  const int bulk_ok = (a.na == 0 || (al16(a.A) && (a.lda & 1) == 0)) && (a.nb == 0 || (al16(a.Bm) && (a.ldb & 1) == 0)) &&
                      (a.bscale == nullptr || al16(a.bscale));
  if (f64)
    k_dfgemm_tc<true><<<blocks, kTcThreads, kTcSmem, st>>>(a, bdig, fexp, kp, bulk_ok, err);
  else
    k_dfgemm_tc<false><<<blocks, kTcThreads, kTcSmem, st>>>(a, bdig, fexp, kp, bulk_ok, err);
  return cudaGetLastError();
}

}  // namespace rk
