// Fused Arnoldi inner products of the FP64 basis on the tcgen05 tensor cores:
// out = [Q^T p (nq), Q^T w (nq), p^T p, p^T w, w^T w] (Algorithm 3, the
// projections onto [C V_j] of one delayed-reorthogonalisation step), with
// every product exact and FP64-level accumulation.
//
// Y = [Q p w] (ncol = nq + 2 <= 64 FP64 columns) is cut, per column and per
// block of 64 rows, into seven unsigned base-256 digits against a power of
// two: with emax the largest exponent field of the column over the block and
// E = emax - 1022 (so |y| < 2^E there), y = sign 2^(E-56) sum_i d_i 256^(6-i)
// + (bits below 2^(E-56), truncated), 0 <= d_i <= 255, taken from the
// IEEE-754 bits with integer operations (every bit of y kept when its
// exponent is within 3 of emax). BF16 holds each digit exactly, a digit
// product is an integer below 2^16, and a 64-row sum of them stays below
// 2^22, so the FP32 accumulation in TMEM is exact. For digit planes i of Y
// and j of v in {p, w}: D_ij = sum_k d_i(y_k) d_j(v_k) over the block, and
//   y^T v (block) = 2^(Ey + Ev - 112) sum_L T_L 256^(12-L),  T_L = sum_{i+j=L} D_ij,
// levels L <= 8 kept (the rest lies below 2^-60 of the block's scale). The
// level sums are combined exactly in 64-bit integers (hi = T_0..T_4,
// lo = T_5..T_8), converted and scaled into an FP64 running sum per (y, v):
// two roundings per block. The truncation of Y to 56 bits bounds the error by
// 2^-55 (max|y| sum|v| + max|v| sum|y|) per block, below FP64's own
// accumulation error.
//
// MMA layout (kind::f16, BF16 digits, FP32 accumulation, both operands
// K-major in shared memory): A rows r = i ncol + c hold plane i of column c
// (7 ncol rows, M = 128 per MMA, up to 4 MMAs); B rows n = 7 v + j hold plane
// j of p (v = 0) and w (v = 1) (N = 16, rows 14-15 zero); K = the 64 rows of
// the block in 4 steps of 16. D_m (128 lanes x 16 columns) = A_m B^T.
//
// One block per SM over a contiguous range of 64-row blocks (deterministic
// for a given n). Warps: 8 producers (each: columns 4g..4g+3 x 8 row chunks,
// one lane per (column, chunk of 8 rows); global loads one block ahead in
// registers, the column's exponent by shuffles, the digits written as 16-byte
// core-matrix rows into one of two digit buffers), one MMA issuer, and 4
// drain warps (one per TMEM lane quarter) that read the accumulators of the
// previous block, convert and regroup them through shared memory by (column,
// v), and update the running sums, one (column, v) pair per thread. A block's
// partials go to `part`; the last block to finish sums them in block order.
#include <cuda_bf16.h>

#include "rk_internal.h"
#include "rk_async.cuh"
#include "rk_device.cuh"
#include "rk_tcgen05.cuh"

namespace rk {

namespace {

constexpr int kTdRows = 64;                       // rows per block = MMA K per block
constexpr int kTdMaxCols = 64;                    // ncol = nq + 2 <= 64
constexpr int kTdPlanes = 7;                      // digits per value
constexpr int kTdProd = 8;                        // producer warps
constexpr int kTdDrain = 4;                       // drain warps
constexpr int kTdThreads = 32 * (kTdProd + 1 + kTdDrain);
constexpr int kTdIssuer = kTdProd;                // warp index of the MMA issuer
constexpr int kTdKg = kTdRows / 8;                // core-matrix columns along K
constexpr int kTdARowsMax = 512;                  // round_up(7 * 64, 128)
constexpr int kTdABytes = kTdARowsMax * kTdRows * 2;  // 64 KB per digit buffer
constexpr int kTdBBytes = 16 * kTdRows * 2;           // 2 KB
constexpr int kTdAcc = 64;                        // TMEM columns per accumulator buffer (4 MMAs x 16)
constexpr int kTdTmem = 128;                      // two accumulator buffers
constexpr size_t kTdSmem = 2 * (size_t)kTdABytes + 2 * (size_t)kTdBBytes +
                           (size_t)kTdMaxCols * 2 * kTdPlanes * kTdPlanes * sizeof(int) + 1024;

// element offset of (row, k) in a K-major canonical operand of kTdKg 8-wide
// core-matrix columns along K (8 x 8 core matrices of 128 bytes)
__device__ __forceinline__ int td_off(int row, int k) {
  return (((row >> 3) * kTdKg + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

// the biased exponent field (0 for zeros and subnormals, which count as 0)
__device__ __forceinline__ int td_expbits(double x) {
  return (int)((unsigned)(__double_as_longlong(x) >> 52) & 0x7ffu);
}

// |y| 2^(56-E) truncated to an integer (< 2^56) as (lo, hi) words, E = emax - 1022
__device__ __forceinline__ void td_fixed56(double y, int emax, unsigned& lo, unsigned& hi) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const int eb = (int)((b >> 52) & 0x7ffu);
  unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;
  const int sh = eb - emax + 3;  // <= 3
  if (eb == 0 || sh <= -56)
    m = 0ull;
  else if (sh >= 0)
    m <<= sh;
  else
    m >>= -sh;
  lo = (unsigned)m;
  hi = (unsigned)(m >> 32);
}

// digit byte `sel` of (lo, hi) (0 = lowest) as a signed FP32 value: the
// byte placed in the mantissa of 2^23 (sign from `mag`), minus 2^23
__device__ __forceinline__ float td_digit(unsigned lo, unsigned hi, int byte, unsigned mag, float off) {
  const unsigned src = byte < 4 ? lo : hi;
  const unsigned sel = (unsigned)(byte & 3) | 0x7650u;  // byte of src, then bytes 1-3 of mag
  return __uint_as_float(__byte_perm(src, mag, sel)) + off;
}

// two digits (integers of at most 8 bits, so the low 16 bits of their FP32
// encodings are zero) as a BF16 pair, lo first
__device__ __forceinline__ uint32_t td_pack(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// exact FP32 integer value (|v| < 2^22) to int
__device__ __forceinline__ int td_int(float v) {
  return __float_as_int(v + 12582912.0f) - 0x4B400000;
}

// 2^e as a double for e in the normal range, else 0 / inf by ldexp
__device__ __forceinline__ double td_pow2(int e) {
  if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(1.0, e);
}

__global__ void __launch_bounds__(kTdThreads, 1) k_dots2_tc(F64Dots2Args a, int nmma) {
  if (a.skip_flag != nullptr && *a.skip_flag != 0) return;
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sA = tsm;                                    // [2][kTdABytes] digits of Y
  unsigned char* sB = tsm + 2 * kTdABytes;                    // [2][kTdBBytes] digits of p, w
  int* dr = reinterpret_cast<int*>(sB + 2 * kTdBBytes);        // [ncol][2][7][7] block sums D_ij
  __shared__ __align__(8) uint64_t full[2], freeb[2], tfull[2], tfree[2], exready[4], done;
  __shared__ uint32_t tslot;
  __shared__ int ex[4][kTdMaxCols];
  __shared__ int lastflag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nq = a.nq, ncol = nq + 2;
  const int64_t nblk = (a.n + kTdRows - 1) / kTdRows;
  const int64_t b0 = nblk * blockIdx.x / gridDim.x, b1 = nblk * (blockIdx.x + 1) / gridDim.x;
  const int nloc = (int)(b1 - b0);
  // B rows 14 and 15 stay zero
  for (int i = tid; i < 2 * 2 * kTdRows; i += kTdThreads) {
    const int buf = i / (2 * kTdRows), rem = i - buf * 2 * kTdRows;
    reinterpret_cast<__nv_bfloat16*>(sB + buf * kTdBBytes)[td_off(14 + rem / kTdRows, rem % kTdRows)] =
        __float2bfloat16(0.f);
  }
  if (warp == 0) tc_alloc(&tslot, kTdTmem);
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&full[b], kTdProd);
      mbar_init(&freeb[b], 1);
      mbar_init(&tfull[b], 1);
      mbar_init(&tfree[b], kTdDrain);
    }
    for (int b = 0; b < 4; ++b) mbar_init(&exready[b], kTdProd);
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
    const int cl = lane >> 3, ch = lane & 7;
    const double* colp[2];
    int cidx[2];
    bool cval[2];
#pragma unroll
    for (int gi = 0; gi < 2; ++gi) {
      const int c = 4 * (warp + kTdProd * gi) + cl;
      cidx[gi] = c;
      cval[gi] = c < ncol;
      colp[gi] = c < nq ? a.Q + (int64_t)c * a.ld : (c == nq ? a.p : a.w);
    }
    const bool g1 = 4 * (warp + kTdProd) < ncol;  // this warp has a second column group
    auto load = [&](int tl, double (&v)[2][8]) {
      const int64_t r0 = (b0 + tl) * kTdRows + 8 * ch;
#pragma unroll
      for (int gi = 0; gi < 2; ++gi) {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[gi][e] = 0.0;
        if (!cval[gi] || (gi == 1 && !g1)) continue;
        const double* src = colp[gi] + r0;
        if (r0 + 8 <= a.n) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const double2 t = __ldg(reinterpret_cast<const double2*>(src) + e);
            v[gi][2 * e] = t.x;
            v[gi][2 * e + 1] = t.y;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (r0 + e < a.n) v[gi][e] = __ldg(src + e);
        }
      }
    };
    double cur[2][8], nxt[2][8];
    if (nloc > 0) load(0, cur);
    for (int tl = 0; tl < nloc; ++tl) {
      if (tl + 1 < nloc) load(tl + 1, nxt);
      const int b = tl & 1;
      if (tl >= 2) wait(&freeb[b], (unsigned)(((tl >> 1) - 1) & 1));  // the MMAs of block tl - 2 are done
      __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(sA + b * kTdABytes);
      __nv_bfloat16* B = reinterpret_cast<__nv_bfloat16*>(sB + b * kTdBBytes);
#pragma unroll
      for (int gi = 0; gi < 2; ++gi) {
        if (gi == 1 && !g1) break;  // warp-uniform
        // the column's largest exponent field over the block (8 lanes)
        int em = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) em = max(em, td_expbits(cur[gi][e]));
        em = max(em, __shfl_xor_sync(0xffffffffu, em, 1));
        em = max(em, __shfl_xor_sync(0xffffffffu, em, 2));
        em = max(em, __shfl_xor_sync(0xffffffffu, em, 4));
        const int c = cidx[gi];
        if (!cval[gi]) continue;
        if (ch == 0) ex[tl & 3][c] = em;
        unsigned lo[8], hi[8], mag[8];
        float off[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          td_fixed56(cur[gi][e], em, lo[e], hi[e]);
          const bool neg = __double_as_longlong(cur[gi][e]) < 0;
          mag[e] = neg ? 0xCB000000u : 0x4B000000u;
          off[e] = neg ? 8388608.0f : -8388608.0f;
        }
#pragma unroll
        for (int i = 0; i < kTdPlanes; ++i) {
          const int byte = 6 - i;  // digit i is byte 6 - i of the 56-bit integer
          uint4 pk;
          pk.x = td_pack(td_digit(lo[0], hi[0], byte, mag[0], off[0]), td_digit(lo[1], hi[1], byte, mag[1], off[1]));
          pk.y = td_pack(td_digit(lo[2], hi[2], byte, mag[2], off[2]), td_digit(lo[3], hi[3], byte, mag[3], off[3]));
          pk.z = td_pack(td_digit(lo[4], hi[4], byte, mag[4], off[4]), td_digit(lo[5], hi[5], byte, mag[5], off[5]));
          pk.w = td_pack(td_digit(lo[6], hi[6], byte, mag[6], off[6]), td_digit(lo[7], hi[7], byte, mag[7], off[7]));
          *reinterpret_cast<uint4*>(A + td_off(i * ncol + c, 8 * ch)) = pk;
          if (c >= nq) *reinterpret_cast<uint4*>(B + td_off(7 * (c - nq) + i, 8 * ch)) = pk;
        }
      }
      fence_async_shared();  // the digits, to the tensor core's proxy
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&full[b]);
        mbar_arrive(&exready[tl & 3]);
      }
#pragma unroll
      for (int gi = 0; gi < 2; ++gi)
#pragma unroll
        for (int e = 0; e < 8; ++e) cur[gi][e] = nxt[gi][e];
    }
  } else if (warp == kTdIssuer) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t a0 = smem_u32(sA), bb0 = smem_u32(sB);
      const uint32_t idesc = tc_idesc_bf16(128, 16);
      for (int tl = 0; tl < nloc; ++tl) {
        const int b = tl & 1;
        wait(&full[b], (unsigned)((tl >> 1) & 1));
        if (tl >= 2) wait(&tfree[b], (unsigned)(((tl >> 1) - 1) & 1));  // block tl - 2 drained
        tc_fence_after_sync();
#pragma unroll
        for (int s = 0; s < kTdRows / 16; ++s) {
          const uint64_t bd = tc_smem_desc(bb0 + b * kTdBBytes + s * 256, 128, kTdKg * 128);
          for (int m = 0; m < nmma; ++m) {
            const uint64_t ad = tc_smem_desc(a0 + b * kTdABytes + m * 16 * kTdKg * 128 + s * 256, 128, kTdKg * 128);
            tc_mma_bf16(taddr + b * kTdAcc + m * 16, ad, bd, idesc, s > 0 ? 1u : 0u);
          }
        }
        tc_commit(&freeb[b]);
        tc_commit(&tfull[b]);
      }
      tc_commit(&done);
      if (!mbar_wait_bounded(&done, 0u)) ok = false;  // every MMA has completed before TMEM is freed
    }
  } else {
    // ------------------------------------------------------------ drain
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int d = tid - 32 * (kTdProd + 1);  // 0..127
    const int pc = d >> 1, pv = d & 1;
    const bool own = d < 2 * ncol;
    double acc = 0.0;
    for (int tl = 0; tl < nloc; ++tl) {
      const int b = tl & 1;
      wait(&tfull[b], (unsigned)((tl >> 1) & 1));
      wait(&exready[tl & 3], (unsigned)((tl >> 2) & 1));
      tc_fence_after_sync();
      for (int m = 0; m < nmma; ++m) {
        float v[16];
        tc_load16(taddr + ((uint32_t)(32 * q) << 16) + b * kTdAcc + m * 16, v);
        const int r = 128 * m + 32 * q + lane;
        const int i = r / ncol, c = r - i * ncol;
        if (i < kTdPlanes) {
#pragma unroll
          for (int vv = 0; vv < 2; ++vv)
#pragma unroll
            for (int j = 0; j < kTdPlanes; ++j) dr[((c * 2 + vv) * 7 + i) * 7 + j] = td_int(v[vv * 7 + j]);
        }
      }
      tc_fence_before_sync();
      named_barrier_sync(1, 32 * kTdDrain);
      if (own) {
        const int* D = dr + (pc * 2 + pv) * 49;
        long long T[9];
#pragma unroll
        for (int L = 0; L <= 8; ++L) {
          int t = 0;
#pragma unroll
          for (int i = 0; i < kTdPlanes; ++i)
            if (L - i >= 0 && L - i < kTdPlanes) t += D[i * 7 + (L - i)];
          T[L] = t;
        }
        const long long hi = (((T[0] * 256 + T[1]) * 256 + T[2]) * 256 + T[3]) * 256 + T[4];
        const long long lo = ((T[5] * 256 + T[6]) * 256 + T[7]) * 256 + T[8];
        const int ey = ex[tl & 3][pc], ev = ex[tl & 3][nq + pv];
        const int es = ey + ev - 2044;  // Ey + Ev
        acc = fma(__ll2double_rn(hi), td_pow2(es - 48), acc);
        acc = fma(__ll2double_rn(lo), td_pow2(es - 80), acc);
        if (ey == 2047 || ev == 2047) acc = __longlong_as_double(0x7ff8000000000000ll);  // Inf / NaN operand
      }
      named_barrier_sync(1, 32 * kTdDrain);
      if (lane == 0) mbar_arrive(&tfree[b]);
    }
    if (own) {
      const int nout = 2 * nq + 3;
      int idx = -1;
      if (pc < nq)
        idx = pv ? nq + pc : pc;
      else if (pc == nq)
        idx = 2 * nq + pv;
      else if (pv == 1)
        idx = 2 * nq + 2;
      if (idx >= 0) a.part[(int64_t)blockIdx.x * nout + idx] = acc;
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

bool dots2_tc_supported(const F64Dots2Args& a) {
  const char* e = std::getenv("RK_TC_DOTS");  // "1": this engine, else the FP64-pipe kernel
  const bool off = !(e != nullptr && e[0] == '1');
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  return !off && a.n >= 1 && a.nq >= 1 && a.nq + 2 <= kTdMaxCols && al16(a.Q) && (a.ld & 1) == 0 && al16(a.p) &&
         al16(a.w);
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
  const int nmma = (kTdPlanes * (a.nq + 2) + 127) / 128;
  k_dots2_tc<<<(int)g, kTdThreads, kTdSmem, st>>>(a, nmma);
  return cudaGetLastError();
}

}  // namespace rk
