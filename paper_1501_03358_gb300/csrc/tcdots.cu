// Fused Arnoldi inner products of the FP64 basis on the tcgen05 tensor cores:
// out = [Q^T p (nq), Q^T w (nq), p^T p, p^T w, w^T w] (Algorithm 3, the
// projections onto [C V_j] of one delayed-reorthogonalisation step), with
// every product exact and the sums kept in 128-bit integers.
//
// Y = [Q p w] (ncol = nq + 2 <= 64 FP64 columns) is cut, per column and per
// block of 32 rows, into seven unsigned base-256 digits against a power of
// two: with emax the largest exponent field of the column over the block and
// E = emax - 1022 (so |y| < 2^E there), y = sign 2^(E-56) sum_i d_i 256^(6-i)
// + (bits below 2^(E-56), truncated), 0 <= d_i <= 255, taken from the
// IEEE-754 bits with integer operations (every bit of y kept when its
// exponent is within 3 of emax). FP16 holds each digit exactly, a digit
// product is an integer below 2^16, and a 32-row sum of them stays below
// 2^21, so the FP32 accumulation in TMEM is exact. For digit planes i of Y
// and j of v in {p, w}: D_ij = sum_k d_i(y_k) d_j(v_k) over the block, and
//   y^T v (block) = 2^(Ey + Ev - 112) sum_L T_L 256^(12-L),  T_L = sum_{i+j=L} D_ij.
// Levels L <= 9 are kept (the rest lies below 2^-70 of the block's scale)
// and summed exactly as a 128-bit integer with a power-of-two scale; blocks
// are added into a 128-bit running sum whose scale follows the largest block
// (bits below 2^-88 of a block's scale may be shifted out). The truncation of
// Y to 56 bits bounds the error by 2^-55 (max|y| sum|v| + max|v| sum|y|) per
// block; one FP64 rounding per block partial and the fixed-order FP64 sum of
// the block partials follow.
//
// MMA layout (kind::f16, FP16 digits, FP32 accumulation, both operands
// K-major in shared memory): A rows 64 i + c hold plane i of column c, so MMA
// m (M = 128) covers planes 2m and 2m + 1 of every column and TMEM lane L
// holds column L mod 64, plane 2m + L / 64; B rows 7 v + j hold plane j of p
// (v = 0) and w (v = 1) (N = 16, rows 14-15 zero); K = the 32 rows of the
// block in 2 steps of 16. D_m (128 lanes x 16 columns) = A_m B^T.
//
// One block per SM over a contiguous range of 32-row blocks (deterministic
// for a given n), four blocks in flight and eight between MMA and drain. Warps:
// - a loader (one thread): each block of Y as one tiled tensor copy of Q's
//   32 x nq box and two of p and w into one of four shared-memory stages,
//   zeros past the last row;
// - 16 producers in two sets of 8 taking alternate blocks: lane l of set warp
//   g takes column 8 g + l / 4, rows 8 (l % 4) .. +7, reads its 8 values from
//   the stage, finds the column's exponent by shuffles and writes each digit
//   plane as one 16-byte core-matrix row (two FP16 digits per byte permute,
//   mask and half2 add) into one of four digit buffers;
// - one MMA issuer (8 MMAs per block into one of eight TMEM accumulators);
// - 4 drain warps (one per TMEM lane quarter): each thread reads its lane's
//   64 accumulator values, forms its planes' level sums and adds them into
//   its two 128-bit running sums, with no shared memory or block barrier.
// At the end the two threads of a column (planes of either parity) add their
// sums and round once to FP64 into `part`; the last block to finish sums the
// blocks' partials in block order.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

#include "rk_internal.h"
#include "rk_async.cuh"
#include "rk_device.cuh"
#include "rk_tcgen05.cuh"

namespace rk {

namespace {

constexpr int kTdRows = 32;                       // rows per block = MMA K per block
constexpr int kTdMaxCols = 64;                    // ncol = nq + 2 <= 64
constexpr int kTdPlanes = 7;                      // digits per value
constexpr int kTdBuf = 4;                         // stages and digit buffers (blocks in flight)
constexpr int kTdAccBuf = 8;                      // TMEM accumulators (blocks between MMA and drain)
constexpr int kTdExDepth = 16;                    // exponent slots (see the producers)
constexpr int kTdSetWarps = 8;                    // producer warps per set (8 columns each)
constexpr int kTdProd = 2 * kTdSetWarps;          // producer warps: two sets, alternate blocks
constexpr int kTdIssuer = kTdProd;                // warp index of the MMA issuer
constexpr int kTdDrain = 4;                       // drain warps (after the issuer)
constexpr int kTdLoader = kTdProd + 1 + kTdDrain;  // warp index of the tensor-copy loader
constexpr int kTdThreads = 32 * (kTdLoader + 1);
constexpr int kTdKg = kTdRows / 8;                // core-matrix columns along K
constexpr int kTdABytes = 512 * kTdRows * 2;      // 32 KB: 4 MMAs x 128 rows
constexpr int kTdBBytes = 16 * kTdRows * 2;       // 1 KB
constexpr int kTdStage = kTdMaxCols * kTdRows * 8;  // 16 KB: one block of Y in FP64
constexpr int kTdAcc = 64;                        // TMEM columns per accumulator (4 MMAs x 16)
constexpr int kTdTmem = kTdAccBuf * kTdAcc;       // 512
constexpr size_t kTdSmem = kTdBuf * ((size_t)kTdABytes + kTdBBytes + kTdStage);

// element offset of (row, k) in a K-major canonical operand of kTdKg 8-wide
// core-matrix columns along K (8 x 8 core matrices of 128 bytes)
__device__ __forceinline__ int td_off(int row, int k) {
  return (((row >> 3) * kTdKg + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

// the biased exponent field (0 for zeros and subnormals, which count as 0)
__device__ __forceinline__ int td_expbits(double x) {
  return (int)((unsigned)(__double_as_longlong(x) >> 52) & 0x7ffu);
}

// |y| 2^(56-E) truncated to an integer (< 2^56) as (lo, hi) words, E = emax - 1022:
// the 53-bit significand moved up 3 bits, then down by emax - eb (zeros and
// subnormals give 0), without branches
__device__ __forceinline__ void td_fixed56(double y, int emax, unsigned& lo, unsigned& hi) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const int eb = (int)((b >> 52) & 0x7ffu);
  const unsigned long long m3 = ((b & 0xfffffffffffffull) | 0x10000000000000ull) << 3;
  const int d = emax - eb;  // >= 0
  unsigned long long f = m3 >> (d < 63 ? d : 63);
  f = (eb == 0 || d >= 56) ? 0ull : f;
  lo = (unsigned)f;
  hi = (unsigned)(f >> 32);
}

// Two FP16 digits (byte k of words a and b) as one half2, a's first: the
// bytes go into the low bytes of the two halves, whose high bytes come from
// `mag` (0x64: the half 1024 + d; 0xE4: -(1024 + d)); adding `off` (-1024 or
// +1024 per half) leaves +d or -d exactly.
__device__ __forceinline__ uint32_t td_pair(unsigned a, unsigned b, int k, unsigned mag, __half2 off) {
  const unsigned sel = (unsigned)k * 0x11u + (unsigned)(4 + k) * 0x1100u;  // [a_k, a_k, b_k, b_k]
  const unsigned z = (__byte_perm(a, b, sel) & 0x00ff00ffu) | mag;
  __half2 h;
  __builtin_memcpy(&h, &z, 4);
  h = __hadd2(h, off);
  uint32_t r;
  __builtin_memcpy(&r, &h, 4);
  return r;
}

// exact FP32 integer value (|v| < 2^22) to int
__device__ __forceinline__ int td_int(float v) {
  return __float_as_int(v + 12582912.0f) - 0x4B400000;
}

// a 128-bit value shifted right arithmetically by s >= 0 (0 or -1 for large s)
__device__ __forceinline__ __int128 td_sar(__int128 v, int s) {
  if (s <= 0) return v;
  if (s >= 127) return v < 0 ? (__int128)-1 : (__int128)0;
  return v >> s;
}

// v 2^e as a double (one rounding of the top 64 significant bits, the rest
// truncated: relative error below 2^-52)
__device__ __forceinline__ double td_i128_to_f64(__int128 v, int e) {
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  unsigned __int128 m = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const unsigned long long hi = (unsigned long long)(m >> 64);
  int sh = 0;
  if (hi != 0) {
    sh = 64 - __clzll((long long)hi);  // bits above the low word
    m >>= sh;
  }
  const double r = ldexp(__ull2double_rn((unsigned long long)m), e + sh);
  return neg ? -r : r;
}

// one box of a tiled tensor map into shared memory, completing on `bar`
__device__ __forceinline__ void td_tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void td_tma_1d(void* dst, const CUtensorMap* map, int x, uint64_t* bar) {
  asm volatile("cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2}], [%3];" ::
                   "r"(smem_u32(dst)),
               "l"(map), "r"(x), "r"(smem_u32(bar))
               : "memory");
}

// instruction descriptor of kind::f16 with FP16 A and B, FP32 accumulation,
// both operands K-major, tile M x N
__host__ __device__ constexpr uint32_t td_idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// tmQ: the nq columns of Q (x = row, y = column; box 32 x nq); tmP, tmW: p
// and w (box 32). Rows beyond n arrive as zeros.
__global__ void __launch_bounds__(kTdThreads, 1)
    k_dots2_tc(F64Dots2Args a, const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmP,
               const __grid_constant__ CUtensorMap tmW) {
  if (a.skip_flag != nullptr && *a.skip_flag != 0) return;
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sA = tsm;                                            // [kTdBuf][kTdABytes] digits of Y
  unsigned char* sB = sA + kTdBuf * kTdABytes;                        // [kTdBuf][kTdBBytes] digits of p, w
  double* stg = reinterpret_cast<double*>(sB + kTdBuf * kTdBBytes);  // [kTdBuf][64][32] blocks of Y
  __shared__ __align__(8) uint64_t full[kTdBuf], freeb[kTdBuf], tfull[kTdAccBuf], tfree[kTdAccBuf],
      sfull[kTdBuf], sfree[kTdBuf], exready[kTdExDepth], done;
  __shared__ uint32_t tslot;
  __shared__ int ex[kTdExDepth][kTdMaxCols];
  __shared__ __int128 cA[kTdMaxCols][2];  // the odd-plane threads' sums, their scales and flags
  __shared__ int cE[kTdMaxCols][2], cF[kTdMaxCols][2];
  __shared__ int lastflag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nq = a.nq, ncol = nq + 2;
  const int64_t nblk = (a.n + kTdRows - 1) / kTdRows;
  const int64_t b0 = nblk * blockIdx.x / gridDim.x, b1 = nblk * (blockIdx.x + 1) / gridDim.x;
  const int nloc = (int)(b1 - b0);
  // B rows 14 and 15 stay zero
  for (int i = tid; i < kTdBuf * 2 * kTdRows; i += kTdThreads) {
    const int buf = i / (2 * kTdRows), rem = i - buf * 2 * kTdRows;
    reinterpret_cast<__half*>(sB + buf * kTdBBytes)[td_off(14 + rem / kTdRows, rem % kTdRows)] = __float2half(0.f);
  }
  if (warp == 0) tc_alloc(&tslot, kTdTmem);
  if (tid == 0) {
    for (int b = 0; b < kTdBuf; ++b) {
      mbar_init(&full[b], kTdSetWarps);
      mbar_init(&freeb[b], 1);
      mbar_init(&sfull[b], 1);
      mbar_init(&sfree[b], kTdSetWarps);
    }
    for (int b = 0; b < kTdAccBuf; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tfree[b], kTdDrain);
    }
    for (int b = 0; b < kTdExDepth; ++b) mbar_init(&exready[b], kTdSetWarps);
    mbar_init(&done, 1);
    mbar_init_fence();
  }
  fence_async_shared();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t taddr = tslot;
  bool ok = true;
  // after one wait has given up the others are skipped (the results are then
  // discarded: the error flag is set), so a broken pipeline ends quickly
  auto wait = [&](uint64_t* bar, unsigned parity) { ok = ok && mbar_wait_bounded(bar, parity); };
  if (warp < kTdProd) {
    // ------------------------------------------------------------ producers
    const int set = warp / kTdSetWarps, g = warp % kTdSetWarps;
    const int ch = lane & 3;
    const int c = 8 * g + (lane >> 2);
    const bool cval = c < ncol;
    for (int tl = set; tl < nloc; tl += 2) {
      const int b = tl & (kTdBuf - 1);
      wait(&sfull[b], (unsigned)((tl >> 2) & 1));
      double v[8];
      {
        const double2* src =
            reinterpret_cast<const double2*>(stg + ((size_t)b * kTdMaxCols + (cval ? c : 0)) * kTdRows + 8 * ch);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const double2 t = cval ? src[e] : make_double2(0.0, 0.0);
          v[2 * e] = t.x;
          v[2 * e + 1] = t.y;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sfree[b]);  // the stage may be refilled (block tl + 4)
      // the column's largest exponent field over the block (4 lanes)
      int em = 0;
#pragma unroll
      for (int e = 0; e < 8; ++e) em = max(em, td_expbits(v[e]));
      em = max(em, __shfl_xor_sync(0xffffffffu, em, 1));
      em = max(em, __shfl_xor_sync(0xffffffffu, em, 2));
      // the MMAs of block tl - 4 are done, so its digit buffer is free, and so is
      // this exponent slot (the drain of block tl - 16 ended before the MMAs of
      // block tl - 8 began, which precede those of block tl - 4)
      if (tl >= kTdBuf) wait(&freeb[b], (unsigned)(((tl >> 2) - 1) & 1));
      if (cval && ch == 0) ex[tl & (kTdExDepth - 1)][c] = em;
      if (cval) {
        unsigned lo[8], hi[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) td_fixed56(v[e], em, lo[e], hi[e]);
        unsigned mag[4];
        __half2 off[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const bool sa = __double_as_longlong(v[2 * q]) < 0, sb = __double_as_longlong(v[2 * q + 1]) < 0;
          mag[q] = (sa ? 0xE400u : 0x6400u) | (sb ? 0xE4000000u : 0x64000000u);
          off[q] = __halves2half2(__float2half(sa ? 1024.f : -1024.f), __float2half(sb ? 1024.f : -1024.f));
        }
        __half* A = reinterpret_cast<__half*>(sA + b * kTdABytes);
        __half* B = reinterpret_cast<__half*>(sB + b * kTdBBytes);
#pragma unroll
        for (int i = 0; i < kTdPlanes; ++i) {
          const int k = 6 - i;  // digit i is byte 6 - i of the 56-bit integer
          uint4 pk;
          if (k < 4) {
            pk.x = td_pair(lo[0], lo[1], k, mag[0], off[0]);
            pk.y = td_pair(lo[2], lo[3], k, mag[1], off[1]);
            pk.z = td_pair(lo[4], lo[5], k, mag[2], off[2]);
            pk.w = td_pair(lo[6], lo[7], k, mag[3], off[3]);
          } else {
            pk.x = td_pair(hi[0], hi[1], k - 4, mag[0], off[0]);
            pk.y = td_pair(hi[2], hi[3], k - 4, mag[1], off[1]);
            pk.z = td_pair(hi[4], hi[5], k - 4, mag[2], off[2]);
            pk.w = td_pair(hi[6], hi[7], k - 4, mag[3], off[3]);
          }
          *reinterpret_cast<uint4*>(A + td_off(64 * i + c, 8 * ch)) = pk;
          if (c >= nq) *reinterpret_cast<uint4*>(B + td_off(7 * (c - nq) + i, 8 * ch)) = pk;
        }
      }
      fence_async_shared();  // the digits, to the tensor core's proxy
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&full[b]);
        mbar_arrive(&exready[tl & (kTdExDepth - 1)]);  // phase tl / 16
      }
    }
  } else if (warp == kTdIssuer) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t a0 = smem_u32(sA), bb0 = smem_u32(sB);
      const uint32_t idesc = td_idesc_f16(128, 16);
      for (int tl = 0; tl < nloc; ++tl) {
        const int b = tl & (kTdBuf - 1), ab = tl & (kTdAccBuf - 1);
        wait(&full[b], (unsigned)((tl >> 2) & 1));
        if (tl >= kTdAccBuf) wait(&tfree[ab], (unsigned)(((tl >> 3) - 1) & 1));  // block tl - 8 drained
        tc_fence_after_sync();
#pragma unroll
        for (int s = 0; s < kTdRows / 16; ++s) {
          const uint64_t bd = tc_smem_desc(bb0 + b * kTdBBytes + s * 256, 128, kTdKg * 128);
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const uint64_t ad = tc_smem_desc(a0 + b * kTdABytes + m * 16 * kTdKg * 128 + s * 256, 128, kTdKg * 128);
            tc_mma_bf16(taddr + ab * kTdAcc + m * 16, ad, bd, idesc, s > 0 ? 1u : 0u);
          }
        }
        tc_commit(&freeb[b]);
        tc_commit(&tfull[ab]);
      }
      tc_commit(&done);
      if (!mbar_wait_bounded(&done, 0u)) ok = false;  // every MMA has completed before TMEM is freed
    }
  } else if (warp == kTdLoader) {
    // ------------------------------------------------------------ loader
    if (lane == 0) {
      for (int tl = 0; tl < nloc; ++tl) {
        const int b = tl & (kTdBuf - 1);
        if (tl >= kTdBuf) wait(&sfree[b], (unsigned)(((tl >> 2) - 1) & 1));  // block tl - 4 has been read
        double* sg = stg + (size_t)b * kTdMaxCols * kTdRows;
        const int x = (int)((b0 + tl) * kTdRows);
        fence_async_shared();
        mbar_arrive_expect_tx(&sfull[b], (unsigned)(ncol * kTdRows * 8));
        td_tma_2d(sg, &tmQ, x, 0, &sfull[b]);
        td_tma_1d(sg + nq * kTdRows, &tmP, x, &sfull[b]);
        td_tma_1d(sg + (nq + 1) * kTdRows, &tmW, x, &sfull[b]);
      }
    }
  } else {
    // ------------------------------------------------------------ drain
    const int q = warp & 3;        // TMEM lane quarter of this warp
    const int L = 32 * q + lane;   // TMEM lane: column L mod 64, planes of parity L / 64
    const int h = L >> 6, c = L & 63;
    const bool own = c < ncol;
    __int128 acc[2] = {0, 0};
    int eacc[2] = {0, 0};
    bool has[2] = {false, false}, bad[2] = {false, false};
    for (int tl = 0; tl < nloc; ++tl) {
      const int ab = tl & (kTdAccBuf - 1);
      wait(&tfull[ab], (unsigned)((tl >> 3) & 1));
      wait(&exready[tl & (kTdExDepth - 1)], (unsigned)((tl >> 4) & 1));
      tc_fence_after_sync();
      // T[v][l] = sum over this thread's planes i = 2m + h of D_ij with 2m + j = l
      // (its level is l + h); levels above 9 are not kept. Two MMAs' columns
      // per round of TMEM loads.
      int T[2][10];
#pragma unroll
      for (int vv = 0; vv < 2; ++vv)
#pragma unroll
        for (int l = 0; l < 10; ++l) T[vv][l] = 0;
#pragma unroll
      for (int mp = 0; mp < 2; ++mp) {
        uint32_t r[2][16];
#pragma unroll
        for (int mm = 0; mm < 2; ++mm) {
          const uint32_t ta = taddr + ((uint32_t)(32 * q) << 16) + ab * kTdAcc + (2 * mp + mm) * 16;
          tc_load8_async(ta, r[mm]);
          tc_load8_async(ta + 8, r[mm] + 8);
        }
        tc_wait_load();
#pragma unroll
        for (int mm = 0; mm < 2; ++mm) {
          const int m = 2 * mp + mm;
          if (2 * m + h < kTdPlanes) {
#pragma unroll
            for (int vv = 0; vv < 2; ++vv)
#pragma unroll
              for (int j = 0; j < kTdPlanes; ++j)
                if (2 * m + j < 10) T[vv][2 * m + j] += td_int(__uint_as_float(r[mm][7 * vv + j]));
          }
        }
      }
      // the block's exponents, read before the release below lets the
      // producers of block tl + 8 overwrite their slot
      const int ey = own ? ex[tl & (kTdExDepth - 1)][c] : 0;
      const int ev0 = ex[tl & (kTdExDepth - 1)][nq], ev1 = ex[tl & (kTdExDepth - 1)][nq + 1];
      tc_fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tfree[ab]);  // the accumulator and the slot may be reused
      if (own) {
#pragma unroll
        for (int vv = 0; vv < 2; ++vv) {
          const int ev = vv ? ev1 : ev0;
          if (ey == 2047 || ev == 2047) bad[vv] = true;
          // V = sum_{level <= 9} T_level 256^(9 - level), an exact integer below
          // 2^95, from two 64-bit Horner sums (each below 2^56)
          long long hi = T[vv][0], lo = T[vv][5];
#pragma unroll
          for (int l = 1; l <= 4; ++l) hi = hi * 256 + T[vv][l];
#pragma unroll
          for (int l = 6; l <= 8; ++l) lo = lo * 256 + T[vv][l];
          const __int128 V = h == 0 ? ((__int128)hi << 40) + ((__int128)lo << 8) + T[vv][9]
                                    : ((__int128)hi << 32) + (__int128)lo;
          if (V != 0) {
            const int e = ey + ev - 2044 - 88;  // the block's value is V 2^e
            if (!has[vv]) {
              acc[vv] = V;
              eacc[vv] = e;
              has[vv] = true;
            } else if (e > eacc[vv]) {
              acc[vv] = td_sar(acc[vv], e - eacc[vv]) + V;
              eacc[vv] = e;
            } else {
              acc[vv] += td_sar(V, eacc[vv] - e);
            }
          }
        }
      }
    }
    // the two threads of a column add their sums; one FP64 rounding
    if (own && h == 1) {
#pragma unroll
      for (int vv = 0; vv < 2; ++vv) {
        cA[c][vv] = acc[vv];
        cE[c][vv] = eacc[vv];
        cF[c][vv] = (has[vv] ? 1 : 0) | (bad[vv] ? 2 : 0);
      }
    }
    named_barrier_sync(1, 32 * kTdDrain);
    if (own && h == 0) {
      const int nout = 2 * nq + 3;
#pragma unroll
      for (int vv = 0; vv < 2; ++vv) {
        __int128 s = acc[vv];
        int es = eacc[vv];
        bool hs = has[vv];
        if (cF[c][vv] & 1) {
          const __int128 o = cA[c][vv];
          const int eo = cE[c][vv];
          if (!hs) {
            s = o;
            es = eo;
            hs = true;
          } else if (eo > es) {
            s = td_sar(s, eo - es) + o;
            es = eo;
          } else {
            s += td_sar(o, es - eo);
          }
        }
        double r = hs ? td_i128_to_f64(s, es) : 0.0;
        if (bad[vv] || (cF[c][vv] & 2)) r = __longlong_as_double(0x7ff8000000000000ll);  // Inf / NaN operand
        int idx = -1;
        if (c < nq)
          idx = vv ? nq + c : c;
        else if (c == nq)
          idx = 2 * nq + vv;
        else if (vv == 1)
          idx = 2 * nq + 2;
        if (idx >= 0) a.part[(int64_t)blockIdx.x * nout + idx] = r;
      }
    }
    __threadfence();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  if (warp == 0) tc_dealloc(taddr, kTdTmem);
  if (!ok && a.err != nullptr) atomicExch(a.err, 3);
  // the last block to finish sums the partials in block order
  if (tid == 0) {
    const unsigned t = atomicAdd(a.counter, 1u);
    lastflag = (t == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (lastflag) {
    __threadfence();
    const int nout = 2 * nq + 3;
    for (int idx = tid; idx < nout; idx += kTdThreads) {
      double s = 0.0;
      for (int g = 0; g < (int)gridDim.x; ++g) s += __ldcg(&a.part[(int64_t)g * nout + idx]);
      a.out[idx] = s;
    }
    if (tid == 0) a.counter[0] = 0u;
  }
}

}  // namespace

namespace {

// cuTensorMapEncodeTiled, through the runtime's driver entry point (no link
// against the driver library)
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
    else
      cudaGetLastError();
  });
  return fn;
}

// FP64 columns of `rows` rows, `cols` columns `ld` elements apart, in boxes
// of 32 rows x cols columns (a rank-2 map, or rank 1 for one vector when
// !rank2); zeros beyond the rows
bool encode_cols(CUtensorMap* m, const double* base, int64_t rows, int cols, int64_t ld, bool rank2) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(double)};
  const cuuint32_t box[2] = {(cuuint32_t)kTdRows, (cuuint32_t)cols};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, rank2 ? 2 : 1, const_cast<double*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool dots2_tc_supported(const F64Dots2Args& a) {
  const char* e = std::getenv("RK_TC_DOTS");  // "1": this engine, else the FP64-pipe kernel
  const bool off = !(e != nullptr && e[0] == '1');
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  return !off && a.n >= kTdRows && a.n < (int64_t(1) << 31) && a.nq >= 1 && a.nq + 2 <= kTdMaxCols && al16(a.Q) &&
         (a.ld & 1) == 0 && al16(a.p) && al16(a.w);
}

cudaError_t launch_dots2_tc(const F64Dots2Args& a, cudaStream_t st) {
  static std::atomic<uint64_t> once{0};
  once_per_device(once, [] {
    cudaFuncSetAttribute(k_dots2_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTdSmem);
  });
  const int64_t nblk = (a.n + kTdRows - 1) / kTdRows;
  int64_t g = kNumSM;
  if (g > dots2_f64_rows(a.n)) g = dots2_f64_rows(a.n);  // rows of the partials buffer
  if (g > nblk) g = nblk;
  CUtensorMap tq, tp, tw;
  if (!encode_cols(&tq, a.Q, a.n, a.nq, a.ld, true) || !encode_cols(&tp, a.p, a.n, 1, a.n, false) ||
      !encode_cols(&tw, a.w, a.n, 1, a.n, false))
    return cudaErrorInvalidValue;
  k_dots2_tc<<<(int)g, kTdThreads, kTdSmem, st>>>(a, tq, tp, tw);
  return cudaGetLastError();
}

}  // namespace rk
