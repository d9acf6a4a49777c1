// Single-block kernels on the small problems of the Krylov cycle:
//  - the Givens least-squares update of each Arnoldi step (Algorithms 1
//    and 3, with the in-cycle residual estimate of the note under
//    Algorithm 1) and the cycle's solve for y and z = -B y;
//  - the harmonic Ritz selection of the recycle space (Algorithm 3's
//    recycle update), done entirely on the device:
//      G = Q_G R_G (Householder),  M'' = (Q_G^T F) R_G^{-1},
//      real Schur form of M'' (Hessenberg + Francis double-shift QR),
//      eigenvectors of the k eigenvalues mu = 1/theta of largest modulus,
//      orthonormal basis Q2 of their span, then
//      C <- W_hat (Q_G Q2),   U <- W (R_G^{-1} Q2).
//    With q = R_G p, G^T G p = theta G^T F p is M'' q = (1/theta) q, so the
//    span selected is that of the harmonic Ritz vectors of the k smallest
//    |theta|, and A U = C, C^T C = I hold by construction.
#include <cmath>
#include "rk_solver.h"
#include "rk_device.cuh"
#include "rk_df.cuh"

namespace rk {

namespace {

constexpr int kHRThreads = 128;

// ---------------------------------------------------------------- Arnoldi
// One step of the Arnoldi process (Algorithm 1; Algorithm 3 with
// Q = [C, V]) by classical Gram-Schmidt with delayed
// reorthogonalisation: the stored column j holds p_j, orthogonalised once
// and scaled by an estimate of its norm, and column j+1 holds w = A M^{-1} p_j.
// With Q = [C, v_0 .. v_{j-1}] and dots = [a = Q^T p_j, b = Q^T w, p^T p,
// p^T w, w^T w] from one fused pass:
//   v_j = (p_j - Q a) / alpha,   alpha^2 = p^T p - ||a||^2   (second pass of p_j),
// which completes Hessenberg column j-1 (it gains beta_{j-1} a and
// h_{j,j-1} = beta_{j-1} alpha) and its Givens rotation and residual estimate.
// Then, since A M^{-1} v_j = (w - A M^{-1} Q a) / alpha and ||a|| is at the
// rounding level, w / alpha stands for A M^{-1} v_j: its first-pass
// coefficients are b / alpha against Q and h_jj = (p^T w - a^T b) / alpha^2
// against v_j, and the next pending vector is p_{j+1} = u / beta_j,
// u = w/alpha - Q b/alpha - v_j h_jj, with the Pythagorean estimate
// beta_j^2 = (w^T w - ||b||^2) / alpha^2 - h_jj^2 (any error in beta_j is
// removed at step j+1, which measures p_{j+1}^T p_{j+1}).
// final_pass (cycle end, dots = [a, p^T p]): completes column j-1 and the
// scale of v_j only.
// Sets upd_mode for the update pass: 0 (v_j and p_{j+1}), 1 (v_j only: the
// cycle stops here), 2 (nothing).
__global__ void k_dcgs_coef(SolveState* s, SmallBuffers b, int kc, int j, int final_pass) {
  __shared__ double red[32];
  __shared__ int sh_skip, sh_stop;
  __shared__ double sh_alpha, sh_ia, sh_bprev;
  if (threadIdx.x == 0) {
    sh_skip = s->done;
    if (!sh_skip && !final_pass) s->nspmv += 1;
  }
  __syncthreads();
  if (sh_skip) {
    if (threadIdx.x == 0) s->upd_mode = 2;
    return;
  }
  const int nq = kc + j;
  const double* A = b.dots;
  const double* Bv = b.dots + nq;
  double aa = 0.0, ab = 0.0, bb = 0.0;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const double x = A[q];
    aa = fma(x, x, aa);
    if (!final_pass) {
      const double y = Bv[q];
      ab = fma(x, y, ab);
      bb = fma(y, y, bb);
    }
  }
  aa = block_sum(aa, red);
  if (!final_pass) {
    ab = block_sum(ab, red);
    bb = block_sum(bb, red);
  }
  const int ldh = b.m + 1;
  if (threadIdx.x == 0) {
    const double pp = A[final_pass ? nq : 2 * nq];
    const double al2 = pp - aa;
    const double alpha = (pp > 0.0 && al2 > 1e-28 * pp) ? sqrt(al2) : 0.0;
    sh_alpha = alpha;
    sh_ia = alpha > 0.0 ? 1.0 / alpha : 0.0;
    sh_bprev = s->scal[3];
    b.sv[j] = alpha > 0.0 ? 1.0 : 0.0;
    if (j == 0) b.g[0] *= alpha;  // r = rho p_0 = rho alpha v_0 + rho C a
    sh_stop = 0;
  }
  __syncthreads();
  const double alpha = sh_alpha, ia = sh_ia, bprev = sh_bprev;
  if (j >= 1) {
    const int c = j - 1;
    for (int l = threadIdx.x; l < nq; l += blockDim.x) {
      const double h = fma(bprev, A[l], b.hacc[l]);
      if (l < kc)
        b.B[l + (int64_t)c * b.kmax] = h;
      else
        b.H[(l - kc) + c * ldh] = h;
    }
    for (int l = j + threadIdx.x; l <= b.m; l += blockDim.x) b.H[l + c * ldh] = l == j ? bprev * alpha : 0.0;
    __syncthreads();
    // the rotation chain below is serial: stage its operands in shared memory
    extern __shared__ double gv[];  // column (m + 2) | cs (m) | sn (m)
    double* R = gv;
    double* scs = gv + b.m + 2;
    double* ssn = scs + b.m;
    for (int l = threadIdx.x; l <= c + 1; l += blockDim.x) R[l] = b.H[l + c * ldh];
    for (int i = threadIdx.x; i < c; i += blockDim.x) {
      scs[i] = b.cs[i];
      ssn[i] = b.sn[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // progressive Givens QR of column c; |g_{c+1}| is the residual estimate
      for (int i = 0; i < c; ++i) {
        const double t = scs[i] * R[i] + ssn[i] * R[i + 1];
        R[i + 1] = -ssn[i] * R[i] + scs[i] * R[i + 1];
        R[i] = t;
      }
      double cg = 1.0, sg = 0.0, rr = R[c];
      if (R[c + 1] != 0.0) {
        rr = hypot(R[c], R[c + 1]);
        cg = R[c] / rr;
        sg = R[c + 1] / rr;
      }
      b.cs[c] = cg;
      b.sn[c] = sg;
      R[c] = rr;
      R[c + 1] = 0.0;
      for (int l = 0; l <= c + 1; ++l) b.R[l + c * ldh] = R[l];
      b.g[c + 1] = -sg * b.g[c];
      b.g[c] = cg * b.g[c];
      const double est = fabs(b.g[c + 1]);
      s->est = est;
      s->jj = j;
      if (est <= s->tolabs || alpha == 0.0) {
        s->done = 1;
        sh_stop = 1;
      }
    }
    __syncthreads();
  } else if (threadIdx.x == 0 && alpha == 0.0) {
    s->done = 1;
    s->jj = 0;
    sh_stop = 1;
  }
  __syncthreads();
  if (final_pass || sh_stop) {
    if (threadIdx.x == 0) {
      s->scal[0] = ia;
      s->upd_mode = alpha > 0.0 ? 1 : 2;
    }
    return;
  }
  // first pass of column j
  for (int l = threadIdx.x; l < nq; l += blockDim.x) b.hacc[l] = Bv[l] * ia;
  if (threadIdx.x == 0) {
    const double pw = A[2 * nq + 1], ww = A[2 * nq + 2];
    const double ia2 = ia * ia;
    const double hj = (pw - ab) * ia2;
    const double ref = ww * ia2;
    const double u2 = (ww - bb) * ia2 - hj * hj;
    const double beta = u2 > 1e-20 * ref ? sqrt(u2) : (ref > 0.0 ? sqrt(ref) : 1.0);
    b.hacc[nq] = hj;
    s->scal[0] = ia;
    s->scal[1] = ia / beta;
    s->scal[2] = hj / beta;
    s->scal[3] = beta;
    s->upd_mode = 0;
  }
}

// The cycle's solve: y = R^{-1} g (the Givens-rotated least squares), z = -B y,
// and the coefficients of the solution update. Column-oriented back
// substitution: the reciprocals of the diagonal are formed in parallel,
// then per column one scalar and a parallel update of the right-hand side
// (R and g staged in shared memory); z one thread per row of B.
constexpr int kSolveThreads = 128;
constexpr int kSolveStageMax = 72;  // R staged in shared memory up to m = 72
template <bool STAGED>
__global__ void __launch_bounds__(kSolveThreads) k_cycle_solve(SolveState* s, SmallBuffers b, int kc) {
  extern __shared__ double cs_sm[];  // [R (jj x jj, ld jj)] | g' (jj) | 1/r_ll (jj) | y (jj)
  const int jj = s->jj;
  const int ldh = b.m + 1;
  const double* R = STAGED ? cs_sm : b.R;
  const int ldr = STAGED ? jj : ldh;
  double* gp = cs_sm + (STAGED ? (size_t)jj * jj : 0);
  double* rinv = gp + jj;
  double* y = rinv + jj;
  if (STAGED)
    for (int t = threadIdx.x; t < jj * jj; t += blockDim.x) {
      const int r = t % jj, c = t / jj;
      cs_sm[t] = r <= c ? b.R[r + c * ldh] : 0.0;
    }
  for (int t = threadIdx.x; t < jj; t += blockDim.x) {
    gp[t] = b.g[t];
    rinv[t] = 1.0 / b.R[t + t * ldh];
  }
  __syncthreads();
  for (int l = jj - 1; l >= 0; --l) {
    const double yl = gp[l] * rinv[l];
    for (int i = threadIdx.x; i < l; i += blockDim.x) gp[i] = fma(-R[i + (int64_t)l * ldr], yl, gp[i]);
    if (threadIdx.x == 0) y[l] = yl;
    __syncthreads();
  }
  for (int q = threadIdx.x; q < kc; q += blockDim.x) {
    double z = 0.0;
    for (int l = 0; l < jj; ++l) z = fma(b.B[q + (int64_t)l * b.kmax], y[l], z);
    b.xcoef[q] = -z;  // z = -B y
  }
  for (int l = threadIdx.x; l < jj; l += blockDim.x) {
    b.y[l] = y[l];
    b.xcoef[kc + l] = b.sv[l] * y[l];
  }
}

// ------------------------------------------------------------ harmonic Ritz
struct HRWork {
  double* G;   // (n+1) x n  -> reflectors below the diagonal, R_G above
  double* F;   // (n+1) x n  -> Q_G^T F, later Z * X
  double* M;   // n x n      -> Schur form T
  double* Z;   // n x n      -> Schur vectors
  double* X;   // n x n      -> selected eigenvectors, then Q2
  double* tau; // n
  double* v;   // n + 1
  double* wr;  // n
  double* wi;  // n
  int* sel;    // n + 1 (selected start index; -1 end), then n flags
};

__device__ HRWork hr_carve(double* base, int n) {
  HRWork w;
  double* p = base;
  w.G = p; p += (size_t)(n + 1) * n;
  w.F = p; p += (size_t)(n + 1) * n;
  w.M = p; p += (size_t)n * n;
  w.Z = p; p += (size_t)n * n;
  w.X = p; p += (size_t)n * n;
  w.tau = p; p += n;
  w.v = p; p += n + 1;
  w.wr = p; p += n;
  w.wi = p; p += n;
  w.sel = (int*)p;
  return w;
}

// Householder vector for x[0..len): on return v[0] = 1, v[1..] scaled, beta
// the new leading entry, tau the coefficient (I - tau v v^T). Block-wide.
__device__ void house(const double* x, int len, double* v, double* beta_out, double* tau_out, double* red) {
  double ss = 0.0;
  for (int i = threadIdx.x + 1; i < len; i += blockDim.x) ss = fma(x[i], x[i], ss);
  const double sig = block_sum(ss, red);
  const double alpha = x[0];
  __syncthreads();
  if (sig == 0.0) {
    for (int i = threadIdx.x; i < len; i += blockDim.x) v[i] = i == 0 ? 1.0 : 0.0;
    if (threadIdx.x == 0) {
      *beta_out = alpha;
      *tau_out = 0.0;
    }
  } else {
    const double nrm = sqrt(alpha * alpha + sig);
    const double beta = alpha <= 0.0 ? nrm : -nrm;
    const double v0 = alpha - beta;
    for (int i = threadIdx.x; i < len; i += blockDim.x) v[i] = i == 0 ? 1.0 : x[i] / v0;
    if (threadIdx.x == 0) {
      *beta_out = beta;
      *tau_out = (beta - alpha) / beta;
    }
  }
  __syncthreads();
}

// A(r0 + i, c) -= tau * v_i * (v^T A(r0:r0+len, c)) for columns c in [c0, c1).
__device__ void apply_left(double* A, int ld, int r0, int len, int c0, int c1, const double* v, double tau) {
  if (tau == 0.0) return;
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    double* col = A + (int64_t)c * ld + r0;
    double w = 0.0;
    for (int i = 0; i < len; ++i) w = fma(v[i], col[i], w);
    w *= tau;
    for (int i = 0; i < len; ++i) col[i] = fma(-w, v[i], col[i]);
  }
}

// Complex helpers
struct cplx { double re, im; };
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  const double s = fabs(b.re) + fabs(b.im);
  const double br = b.re / s, bi = b.im / s;
  const double d = br * br + bi * bi;
  return {(a.re * br + a.im * bi) / (d * s), (a.im * br - a.re * bi) / (d * s)};
}

// 3- or 2-vector Householder reflector in double-float (one thread):
// (I - tau v v^T) [x y z]^T = [beta 0 0]^T with v = [1, v1, v2].
// The vector is first scaled by a power of two (exact) so that its largest
// component is in [0.5, 1): the bulge entries become tiny as the iteration
// converges, and their squares would leave the FP32 exponent range.
__device__ void house_small_df(float2 x, float2 y, float2 z, int len, float2* v, float2* tau) {
  const bool tail_zero = y.x == 0.f && (len == 2 || z.x == 0.f);
  const float mx = fmaxf(fabsf(x.x), fmaxf(fabsf(y.x), len == 3 ? fabsf(z.x) : 0.f));
  v[0] = make_float2(1.f, 0.f);
  if (!(mx > 0.f) || tail_zero) {
    v[1] = v[2] = make_float2(0.f, 0.f);
    *tau = make_float2(0.f, 0.f);
    return;
  }
  int ex;
  frexpf(mx, &ex);
  const float sc = ldexpf(1.f, -ex);
  x = make_float2(x.x * sc, x.y * sc);
  y = make_float2(y.x * sc, y.y * sc);
  z = make_float2(z.x * sc, z.y * sc);
  float2 ss = df_mul(x, x);
  ss = df_fma(y, y, ss);
  if (len == 3) ss = df_fma(z, z, ss);
  const float2 nrm = df_sqrt_fast(ss);
  const float2 beta = x.x <= 0.f ? nrm : df_neg(nrm);
  const float2 v0 = df_sub(x, beta);
  // the two quotients are independent (their chains overlap)
  const float2 rv0 = df_div_fast(make_float2(1.f, 0.f), v0);
  *tau = df_div_fast(df_sub(beta, x), beta);
  v[1] = df_mul(y, rv0);
  v[2] = len == 3 ? df_mul(z, rv0) : make_float2(0.f, 0.f);
}

// h <- (I - tau v v^T) h for a 3-vector (v0 = 1) or a 2-vector (v2 = 0)
__device__ __forceinline__ void refl3_df(float2& h0, float2& h1, float2& h2, float2 v1, float2 v2, float2 tau) {
  float2 t = df_fma(v1, h1, h0);
  t = df_fma(v2, h2, t);
  const float2 ww = df_mul(tau, t);
  h0 = df_sub(h0, ww);
  h1 = df_fma(df_neg(ww), v1, h1);
  h2 = df_fma(df_neg(ww), v2, h2);
}
__device__ __forceinline__ void refl2_df(float2& h0, float2& h1, float2 v1, float2 tau) {
  const float2 ww = df_mul(tau, df_fma(v1, h1, h0));
  h0 = df_sub(h0, ww);
  h1 = df_fma(df_neg(ww), v1, h1);
}

// Block sum of per-thread double-float values; every thread gets the result.
__device__ float2 block_df_sum(float2 v, float2* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = df_warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float2 t = red[0];
  for (int q = 1; q < nw; ++q) t = df_add(t, red[q]);
  return t;
}

// Householder reduction to upper Hessenberg form H = Z^T M Z in double-float
// (the reflectors of column c act on rows/columns c+1..n-1; Z accumulates
// them). H has leading dimension ldh, Z leading dimension n; v is a scratch
// vector of n double-float values. Block-wide; the Z updates run on threads
// 64.. while threads 0..63 update the rows of H.
__device__ void hessenberg_df(float2* H, int ldh, float2* Z, int n, float2* v) {
  __shared__ float2 red2[32];
  __shared__ float2 hb[2];  // beta, tau
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int c = 0; c + 2 < n; ++c) {
    const int len = n - c - 1;
    float2* x = H + (int64_t)c * ldh + c + 1;
    float sh = 0.f, sl = 0.f;
    for (int i = tid + 1; i < len; i += bd) df_mac(sh, sl, x[i].x, x[i].y, x[i].x, x[i].y);
    const float2 sig = block_df_sum(make_float2(sh, sl), red2);
    const float2 alpha = x[0];
    if (!(sig.x > 0.f)) {
      for (int i = tid; i < len; i += bd) v[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
      if (tid == 0) {
        hb[0] = alpha;
        hb[1] = make_float2(0.f, 0.f);
      }
    } else {
      const float2 nrm = df_sqrt_fast(df_fma(alpha, alpha, sig));
      const float2 beta = alpha.x <= 0.f ? nrm : df_neg(nrm);
      const float2 rv0 = df_div_fast(make_float2(1.f, 0.f), df_sub(alpha, beta));
      for (int i = tid; i < len; i += bd) v[i] = i == 0 ? make_float2(1.f, 0.f) : df_mul(x[i], rv0);
      if (tid == 0) {
        hb[0] = beta;
        hb[1] = df_div_fast(df_sub(beta, alpha), beta);
      }
    }
    __syncthreads();
    const float2 tau = hb[1];
    if (tau.x != 0.f) {
      // from the left: columns c..n-1, rows c+1..n-1
      for (int j = c + tid; j < n; j += bd) {
        float2* col = H + (int64_t)j * ldh + c + 1;
        float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
        int i = 0;
        for (; i + 1 < len; i += 2) {
          df_mac(ah, al, v[i].x, v[i].y, col[i].x, col[i].y);
          df_mac(bh, bl, v[i + 1].x, v[i + 1].y, col[i + 1].x, col[i + 1].y);
        }
        if (i < len) df_mac(ah, al, v[i].x, v[i].y, col[i].x, col[i].y);
        const float2 ww = df_neg(df_mul(tau, df_add(make_float2(ah, al), make_float2(bh, bl))));
        for (int i2 = 0; i2 < len; ++i2) col[i2] = df_fma(ww, v[i2], col[i2]);
      }
      __syncthreads();
      // from the right: rows 0..n-1 of H (threads 0..63) and of Z (threads 64..)
      const bool zpart = tid >= 64;
      float2* A = zpart ? Z : H;
      const int lda = zpart ? n : ldh;
      const int t0 = zpart ? tid - 64 : tid, ts = zpart ? bd - 64 : 64;
      for (int r = t0; r < n; r += ts) {
        float2* row = A + r + (int64_t)(c + 1) * lda;
        float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
        int i = 0;
        for (; i + 1 < len; i += 2) {
          df_mac(ah, al, row[(int64_t)i * lda].x, row[(int64_t)i * lda].y, v[i].x, v[i].y);
          df_mac(bh, bl, row[(int64_t)(i + 1) * lda].x, row[(int64_t)(i + 1) * lda].y, v[i + 1].x, v[i + 1].y);
        }
        if (i < len) df_mac(ah, al, row[(int64_t)i * lda].x, row[(int64_t)i * lda].y, v[i].x, v[i].y);
        const float2 ww = df_neg(df_mul(tau, df_add(make_float2(ah, al), make_float2(bh, bl))));
        for (int i2 = 0; i2 < len; ++i2) row[(int64_t)i2 * lda] = df_fma(ww, v[i2], row[(int64_t)i2 * lda]);
      }
      __syncthreads();
    }
    for (int i = tid; i < len; i += bd) x[i] = i == 0 ? hb[0] : make_float2(0.f, 0.f);
    __syncthreads();
  }
}

// Francis double-shift QR (implicit, bulge chasing with 3x3 reflectors;
// exceptional shifts at iterations 10 and 20 of one eigenvalue; deflation
// when |h_{l,l-1}| <= 2^-47 (|h_{l-1,l-1}| + |h_ll|); 2x2 blocks with real
// eigenvalues split by a rotation) on Hd (n x n Hessenberg, DF), with the
// transformations accumulated into Zd. hn: max |h_ij|. Block-wide;
// eigenvalues to wr, wi (FP64). On more than 40 n iterations *sfail is set.
__device__ void francis_df(float2* Hd, int ldh, float2* Zd, int n, double* wr, double* wi, float hn, int* su,
                           int* sl, int* siter, int* stotal, int* sfail) {
  __shared__ float2 v3[3], tau3, rot[2], fxyz[3];
  __shared__ int c_real;
  const float eps = 7.105427357601002e-15f;    // 2^-47
  const float floor_abs = 1.4210854715202004e-14f * hn;  // 2^-46 max |h_ij|
  const int tid = threadIdx.x;
#define HD(i, j) Hd[(i) + (int64_t)(j) * ldh]
#define ZD(i, j) Zd[(i) + (int64_t)(j) * n]
  while (true) {
    __syncthreads();
    const int u = *su;
    if (u < 0 || *sfail) break;
    if (tid == 0) {
      int l = u;
      while (l > 0) {
        // relative to the neighbouring diagonal, with an absolute floor at the
        // double-float rounding level of the whole matrix (a subdiagonal next
        // to eigenvalues near zero cannot drop below that noise)
        const float h = fabsf(HD(l, l - 1).x);
        const float sc = fabsf(HD(l - 1, l - 1).x) + fabsf(HD(l, l).x);
        if (h <= eps * sc || h <= floor_abs) break;
        --l;
      }
      if (l > 0) HD(l, l - 1) = make_float2(0.f, 0.f);
      *sl = l;
    }
    __syncthreads();
    const int l = *sl;
    if (l == u) {  // 1 x 1 block
      if (tid == 0) {
        wr[u] = df_to_double(HD(u, u));
        wi[u] = 0.0;
        *su = u - 1;
        *siter = 0;
      }
      continue;
    }
    if (l == u - 1) {  // 2 x 2 block: split if real (FP64 rotation), record the pair if complex
      if (tid == 0) {
        const double a = df_to_double(HD(u - 1, u - 1)), bb = df_to_double(HD(u - 1, u));
        const double c = df_to_double(HD(u, u - 1)), d = df_to_double(HD(u, u));
        const double p = 0.5 * (a - d);
        const double disc = p * p + bb * c;
        if (disc >= 0.0) {
          const double sq = sqrt(disc);
          const double zz = p + (p >= 0.0 ? sq : -sq);
          double cs = 1.0, sn = 0.0;
          if (zz != 0.0 || c != 0.0) {
            const double r = hypot(zz, c);
            cs = zz / r;
            sn = c / r;
          }
          rot[0] = df_make(cs);
          rot[1] = df_make(sn);
          c_real = 1;
        } else {
          c_real = 0;
          wr[u - 1] = 0.5 * (a + d);
          wr[u] = 0.5 * (a + d);
          wi[u - 1] = sqrt(-disc);
          wi[u] = -sqrt(-disc);
        }
      }
      __syncthreads();
      if (c_real) {
        const float2 cs = rot[0], sn = rot[1];
        for (int j = u - 1 + tid; j < n; j += blockDim.x) {
          const float2 h1 = HD(u - 1, j), h2 = HD(u, j);
          HD(u - 1, j) = df_fma(sn, h2, df_mul(cs, h1));
          HD(u, j) = df_fma(cs, h2, df_neg(df_mul(sn, h1)));
        }
        __syncthreads();
        for (int i = tid; i <= u; i += blockDim.x) {
          const float2 h1 = HD(i, u - 1), h2 = HD(i, u);
          HD(i, u - 1) = df_fma(sn, h2, df_mul(cs, h1));
          HD(i, u) = df_fma(cs, h2, df_neg(df_mul(sn, h1)));
        }
        for (int i = tid; i < n; i += blockDim.x) {
          const float2 z1 = ZD(i, u - 1), z2 = ZD(i, u);
          ZD(i, u - 1) = df_fma(sn, z2, df_mul(cs, z1));
          ZD(i, u) = df_fma(cs, z2, df_neg(df_mul(sn, z1)));
        }
        __syncthreads();
        if (tid == 0) {
          HD(u, u - 1) = make_float2(0.f, 0.f);
          wr[u - 1] = df_to_double(HD(u - 1, u - 1));
          wr[u] = df_to_double(HD(u, u));
          wi[u - 1] = 0.0;
          wi[u] = 0.0;
        }
      }
      if (tid == 0) {
        *su = u - 2;
        *siter = 0;
      }
      continue;
    }
    // Francis double-shift step on the active window [l, u]
    if (tid == 0) {
      *siter += 1;
      *stotal += 1;
      if (*stotal > 40 * n) *sfail = 1;
      float2 sh, th;
      if (*siter == 10 || *siter == 20) {
        const float2 ww = df_add(df_absv(HD(u, u - 1)), u >= 2 ? df_absv(HD(u - 1, u - 2)) : make_float2(0.f, 0.f));
        sh = df_mul(make_float2(1.5f, 0.f), ww);
        th = df_mul(ww, ww);
      } else {
        sh = df_add(HD(u - 1, u - 1), HD(u, u));
        th = df_sub(df_mul(HD(u - 1, u - 1), HD(u, u)), df_mul(HD(u - 1, u), HD(u, u - 1)));
      }
      const float2 hll = HD(l, l), h1l = HD(l + 1, l);
      float2 fx = df_fma(hll, hll, df_mul(HD(l, l + 1), h1l));
      fx = df_add(df_fma(df_neg(sh), hll, fx), th);
      const float2 fy = df_mul(h1l, df_sub(df_add(hll, HD(l + 1, l + 1)), sh));
      const float2 fz = (l + 2 <= u) ? df_mul(h1l, HD(l + 2, l + 1)) : make_float2(0.f, 0.f);
      house_small_df(fx, fy, fz, 3, v3, &tau3);
    }
    __syncthreads();
    if (*sfail) break;
    // the bulge chase: each step applies its reflector from the left (rows
    // kk..kk+2) and from the right (columns kk..kk+2, Schur vectors on other
    // warps); the threads that update rows kk+1..kk+3 of column kk publish
    // the new bulge entries in fxyz, and every thread then forms the next
    // reflector itself (same inputs, same result), one barrier per step less
    float2 tau = tau3, v1 = v3[1], v2 = v3[2];
    for (int kk = l; kk <= u - 2; ++kk) {
      if (tau.x != 0.f) {
        const int q = kk > l ? kk - 1 : l;
        for (int j = q + tid; j < n; j += blockDim.x) {
          float2 h0 = HD(kk, j), h1 = HD(kk + 1, j), h2 = HD(kk + 2, j);
          refl3_df(h0, h1, h2, v1, v2, tau);
          HD(kk, j) = h0;
          HD(kk + 1, j) = h1;
          HD(kk + 2, j) = h2;
        }
        __syncthreads();
        const int rmaxi = kk + 3 < u ? kk + 3 : u;
        if (tid < 64) {
          for (int i = tid; i <= rmaxi; i += 64) {
            float2 h0 = HD(i, kk), h1 = HD(i, kk + 1), h2 = HD(i, kk + 2);
            refl3_df(h0, h1, h2, v1, v2, tau);
            HD(i, kk) = h0;
            HD(i, kk + 1) = h1;
            HD(i, kk + 2) = h2;
            if (i > kk) fxyz[i - kk - 1] = h0;
          }
        } else {
          for (int i = tid - 64; i < n; i += (int)blockDim.x - 64) {
            float2 z0 = ZD(i, kk), z1 = ZD(i, kk + 1), z2 = ZD(i, kk + 2);
            refl3_df(z0, z1, z2, v1, v2, tau);
            ZD(i, kk) = z0;
            ZD(i, kk + 1) = z1;
            ZD(i, kk + 2) = z2;
          }
        }
      } else {
        __syncthreads();  // every thread has formed its reflector from fxyz
        if (tid == 0)
          for (int i = 0; i < 3 && kk + 1 + i <= u; ++i) fxyz[i] = HD(kk + 1 + i, kk);
      }
      __syncthreads();
      float2 vv[3];
      if (kk < u - 2)
        house_small_df(fxyz[0], fxyz[1], fxyz[2], 3, vv, &tau);
      else
        house_small_df(fxyz[0], fxyz[1], make_float2(0.f, 0.f), 2, vv, &tau);
      v1 = vv[1];
      v2 = vv[2];
    }
    // final 2-vector reflector on rows / columns u-1, u (formed above)
    {
      if (tau.x != 0.f) {
        const int q = u - 2 >= l ? u - 2 : l;
        for (int j = q + tid; j < n; j += blockDim.x) {
          float2 h0 = HD(u - 1, j), h1 = HD(u, j);
          refl2_df(h0, h1, v1, tau);
          HD(u - 1, j) = h0;
          HD(u, j) = h1;
        }
        __syncthreads();
        if (tid < 64) {
          for (int i = tid; i <= u; i += 64) {
            float2 h0 = HD(i, u - 1), h1 = HD(i, u);
            refl2_df(h0, h1, v1, tau);
            HD(i, u - 1) = h0;
            HD(i, u) = h1;
          }
        } else {
          for (int i = tid - 64; i < n; i += (int)blockDim.x - 64) {
            float2 z0 = ZD(i, u - 1), z1 = ZD(i, u);
            refl2_df(z0, z1, v1, tau);
            ZD(i, u - 1) = z0;
            ZD(i, u) = z1;
          }
        }
      }
    }
    // entries below the subdiagonal are zero by construction
    if (tid == 0) {
      for (int i = l + 2; i <= u; ++i) {
        HD(i, i - 2) = make_float2(0.f, 0.f);
        if (i >= l + 3) HD(i, i - 3) = make_float2(0.f, 0.f);
      }
    }
  }
#undef HD
#undef ZD
}

// A(r, c0 + i) -= tau * (A(r, c0:c0+len) v) v_i for rows r in [r0, r1).
__device__ void apply_right(double* A, int ld, int r0, int r1, int c0, int len, const double* v, double tau) {
  if (tau == 0.0) return;
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    double w = 0.0;
    for (int i = 0; i < len; ++i) w = fma(A[r + (int64_t)(c0 + i) * ld], v[i], w);
    w *= tau;
    for (int i = 0; i < len; ++i) A[r + (int64_t)(c0 + i) * ld] = fma(-w, v[i], A[r + (int64_t)(c0 + i) * ld]);
  }
}

// 3- or 2-vector Householder reflector in FP64 (one thread):
// (I - tau v v^T) [x y z]^T = [beta 0 0]^T with v = [1, v1, v2].
__device__ void house_small_f64(double x, double y, double z, int len, double* v, double* tau) {
  const double nrm = len == 3 ? sqrt(fma(x, x, fma(y, y, z * z))) : sqrt(fma(x, x, y * y));
  v[0] = 1.0;
  if (nrm == 0.0 || (y == 0.0 && (len == 2 || z == 0.0))) {
    v[1] = v[2] = 0.0;
    *tau = 0.0;
    return;
  }
  const double beta = x <= 0.0 ? nrm : -nrm;
  const double v0 = x - beta;
  v[1] = y / v0;
  v[2] = len == 3 ? z / v0 : 0.0;
  *tau = (beta - x) / beta;
}

// Householder reduction to upper Hessenberg form H = Z^T M Z in FP64, in
// place on M (n x n, leading dimension n), Z (n x n) accumulating the
// reflectors; v: n + 1 scratch doubles. Block-wide.
__device__ void hessenberg_f64(double* M, double* Z, int n, double* v, double* red, double* sh_beta, double* sh_tau) {
  for (int c = 0; c + 2 < n; ++c) {
    const int len = n - c - 1;
    double* x = M + (int64_t)c * n + c + 1;
    house(x, len, v, sh_beta, sh_tau, red);
    const double tau = *sh_tau;
    apply_left(M, n, c + 1, len, c, n, v, tau);
    __syncthreads();
    apply_right(M, n, 0, n, c + 1, len, v, tau);
    apply_right(Z, n, 0, n, c + 1, len, v, tau);
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) x[i] = i == 0 ? *sh_beta : 0.0;
    __syncthreads();
  }
}

// Francis double-shift QR in FP64 (implicit, bulge chasing with 3 x 3
// reflectors; exceptional shifts at iterations 10 and 20 of one
// eigenvalue; deflation when |h_{l,l-1}| <= 2^-52 (|h_{l-1,l-1}| + |h_ll|)
// or below 2^-52 max |h_ij|; 2 x 2 blocks with real eigenvalues split by a
// rotation) on H (n x n Hessenberg, leading dimension n) with the
// transformations accumulated into Z. hmax: max |h_ij|. Block-wide;
// eigenvalues to wr, wi. On more than 40 n iterations *sfail is set.
__device__ void francis_f64(double* H, double* Z, int n, double* wr, double* wi, double hmax, int* su, int* sl,
                            int* siter, int* stotal, int* sfail) {
  __shared__ double v3[3], tau3, fxyz[3], rot[2];
  __shared__ int c_real;
  const double eps = 2.220446049250313e-16;  // 2^-52
  const double floor_abs = eps * hmax;
  const int tid = threadIdx.x;
#define HF(i, j) H[(i) + (int64_t)(j) * n]
#define ZF(i, j) Z[(i) + (int64_t)(j) * n]
  while (true) {
    __syncthreads();
    const int u = *su;
    if (u < 0 || *sfail) break;
    if (tid == 0) {
      int l = u;
      while (l > 0) {
        const double h = fabs(HF(l, l - 1));
        const double sc = fabs(HF(l - 1, l - 1)) + fabs(HF(l, l));
        if (h <= eps * sc || h <= floor_abs) break;
        --l;
      }
      if (l > 0) HF(l, l - 1) = 0.0;
      *sl = l;
    }
    __syncthreads();
    const int l = *sl;
    if (l == u) {  // 1 x 1 block
      if (tid == 0) {
        wr[u] = HF(u, u);
        wi[u] = 0.0;
        *su = u - 1;
        *siter = 0;
      }
      continue;
    }
    if (l == u - 1) {  // 2 x 2 block: split if real, record the pair if complex
      if (tid == 0) {
        const double a = HF(u - 1, u - 1), bb = HF(u - 1, u), c = HF(u, u - 1), d = HF(u, u);
        const double p = 0.5 * (a - d);
        const double disc = fma(p, p, bb * c);
        if (disc >= 0.0) {
          const double sq = sqrt(disc);
          const double zz = p + (p >= 0.0 ? sq : -sq);
          double cs = 1.0, sn = 0.0;
          if (zz != 0.0 || c != 0.0) {
            const double r = hypot(zz, c);
            cs = zz / r;
            sn = c / r;
          }
          rot[0] = cs;
          rot[1] = sn;
          c_real = 1;
        } else {
          c_real = 0;
          wr[u - 1] = 0.5 * (a + d);
          wr[u] = 0.5 * (a + d);
          wi[u - 1] = sqrt(-disc);
          wi[u] = -sqrt(-disc);
        }
      }
      __syncthreads();
      if (c_real) {
        const double cs = rot[0], sn = rot[1];
        for (int j = u - 1 + tid; j < n; j += blockDim.x) {
          const double h1 = HF(u - 1, j), h2 = HF(u, j);
          HF(u - 1, j) = cs * h1 + sn * h2;
          HF(u, j) = -sn * h1 + cs * h2;
        }
        __syncthreads();
        for (int i = tid; i <= u; i += blockDim.x) {
          const double h1 = HF(i, u - 1), h2 = HF(i, u);
          HF(i, u - 1) = cs * h1 + sn * h2;
          HF(i, u) = -sn * h1 + cs * h2;
        }
        for (int i = tid; i < n; i += blockDim.x) {
          const double z1 = ZF(i, u - 1), z2 = ZF(i, u);
          ZF(i, u - 1) = cs * z1 + sn * z2;
          ZF(i, u) = -sn * z1 + cs * z2;
        }
        __syncthreads();
        if (tid == 0) {
          HF(u, u - 1) = 0.0;
          wr[u - 1] = HF(u - 1, u - 1);
          wr[u] = HF(u, u);
          wi[u - 1] = 0.0;
          wi[u] = 0.0;
        }
      }
      if (tid == 0) {
        *su = u - 2;
        *siter = 0;
      }
      continue;
    }
    // Francis double-shift step on the active window [l, u]
    if (tid == 0) {
      *siter += 1;
      *stotal += 1;
      if (*stotal > 40 * n) *sfail = 1;
      double s, t;
      if (*siter == 10 || *siter == 20) {
        const double ww = fabs(HF(u, u - 1)) + (u >= 2 ? fabs(HF(u - 1, u - 2)) : 0.0);
        s = 1.5 * ww;
        t = ww * ww;
      } else {
        s = HF(u - 1, u - 1) + HF(u, u);
        t = HF(u - 1, u - 1) * HF(u, u) - HF(u - 1, u) * HF(u, u - 1);
      }
      fxyz[0] = HF(l, l) * HF(l, l) + HF(l, l + 1) * HF(l + 1, l) - s * HF(l, l) + t;
      fxyz[1] = HF(l + 1, l) * (HF(l, l) + HF(l + 1, l + 1) - s);
      fxyz[2] = (l + 2 <= u) ? HF(l + 1, l) * HF(l + 2, l + 1) : 0.0;
    }
    __syncthreads();
    if (*sfail) break;
    for (int kk = l; kk <= u - 2; ++kk) {
      if (tid == 0) house_small_f64(fxyz[0], fxyz[1], fxyz[2], 3, v3, &tau3);
      __syncthreads();
      const double tau = tau3;
      const double v1 = v3[1], v2 = v3[2];
      if (tau != 0.0) {
        const int q = kk > l ? kk - 1 : l;
        for (int j = q + tid; j < n; j += blockDim.x) {
          const double h0 = HF(kk, j), h1 = HF(kk + 1, j), h2 = HF(kk + 2, j);
          const double ww = tau * fma(v2, h2, fma(v1, h1, h0));
          HF(kk, j) = h0 - ww;
          HF(kk + 1, j) = fma(-ww, v1, h1);
          HF(kk + 2, j) = fma(-ww, v2, h2);
        }
        __syncthreads();
        const int rmaxi = kk + 3 < u ? kk + 3 : u;
        for (int i = tid; i <= rmaxi; i += blockDim.x) {
          const double h0 = HF(i, kk), h1 = HF(i, kk + 1), h2 = HF(i, kk + 2);
          const double ww = tau * fma(v2, h2, fma(v1, h1, h0));
          HF(i, kk) = h0 - ww;
          HF(i, kk + 1) = fma(-ww, v1, h1);
          HF(i, kk + 2) = fma(-ww, v2, h2);
        }
        for (int i = tid; i < n; i += blockDim.x) {
          const double h0 = ZF(i, kk), h1 = ZF(i, kk + 1), h2 = ZF(i, kk + 2);
          const double ww = tau * fma(v2, h2, fma(v1, h1, h0));
          ZF(i, kk) = h0 - ww;
          ZF(i, kk + 1) = fma(-ww, v1, h1);
          ZF(i, kk + 2) = fma(-ww, v2, h2);
        }
      }
      __syncthreads();
      if (tid == 0) {
        fxyz[0] = HF(kk + 1, kk);
        fxyz[1] = HF(kk + 2, kk);
        fxyz[2] = kk < u - 2 ? HF(kk + 3, kk) : 0.0;
      }
      __syncthreads();
    }
    // final 2-vector reflector on rows u-1, u
    if (tid == 0) house_small_f64(fxyz[0], fxyz[1], 0.0, 2, v3, &tau3);
    __syncthreads();
    {
      const double tau = tau3;
      const double v1 = v3[1];
      if (tau != 0.0) {
        const int q = u - 2 >= l ? u - 2 : l;
        for (int j = q + tid; j < n; j += blockDim.x) {
          const double h0 = HF(u - 1, j), h1 = HF(u, j);
          const double ww = tau * fma(v1, h1, h0);
          HF(u - 1, j) = h0 - ww;
          HF(u, j) = fma(-ww, v1, h1);
        }
        __syncthreads();
        for (int i = tid; i <= u; i += blockDim.x) {
          const double h0 = HF(i, u - 1), h1 = HF(i, u);
          const double ww = tau * fma(v1, h1, h0);
          HF(i, u - 1) = h0 - ww;
          HF(i, u) = fma(-ww, v1, h1);
        }
        for (int i = tid; i < n; i += blockDim.x) {
          const double h0 = ZF(i, u - 1), h1 = ZF(i, u);
          const double ww = tau * fma(v1, h1, h0);
          ZF(i, u - 1) = h0 - ww;
          ZF(i, u) = fma(-ww, v1, h1);
        }
      }
    }
    __syncthreads();
    // the entries below the subdiagonal that rounding leaves behind
    if (tid == 0) {
      for (int i = l + 2; i <= u; ++i) {
        HF(i, i - 2) = 0.0;
        if (i >= l + 3) HF(i, i - 3) = 0.0;
      }
    }
  }
#undef HF
#undef ZF
}

// Core: G, F already in w.G, w.F (ld n+1). Outputs QC (ld ldqc, n+1 rows),
// PU (ld ldpu, n rows), *knew_out, *status_out (0 ok).
__device__ void hr_core(HRWork w, int n, int k, double* QC, int ldqc, double* PU, int ldpu, int* knew_out,
                        int* status_out, int schur_f64) {
  __shared__ double red[32];
  __shared__ double sh_beta, sh_tau;
  __shared__ int sh_u, sh_l, sh_iter, sh_total, sh_fail, sh_knew;
  const int ldg = n + 1;
  const double eps = 2.220446049250313e-16;

  // ---- 1. Householder QR of G; the same reflectors applied to F.
  for (int c = 0; c < n; ++c) {
    const int len = n + 1 - c;
    double* x = w.G + (int64_t)c * ldg + c;
    house(x, len, w.v, &sh_beta, &sh_tau, red);
    const double tau = sh_tau;
    apply_left(w.G, ldg, c, len, c + 1, n, w.v, tau);
    apply_left(w.F, ldg, c, len, 0, n, w.v, tau);
    __syncthreads();
    // store the reflector below the diagonal
    for (int i = threadIdx.x; i < len; i += blockDim.x) x[i] = i == 0 ? sh_beta : w.v[i];
    if (threadIdx.x == 0) w.tau[c] = tau;
    __syncthreads();
  }
  // ---- 2. M = (Q_G^T F)(0:n, 0:n) R_G^{-1}, row by row.
  if (threadIdx.x == 0) sh_fail = 0;
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    if (!(fabs(w.G[c + (int64_t)c * ldg]) > 1e-300)) sh_fail = 1;
  __syncthreads();
  if (sh_fail) {
    if (threadIdx.x == 0) { *status_out = 1; *knew_out = 0; }
    return;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    for (int c = 0; c < n; ++c) {
      double t = w.F[i + (int64_t)c * ldg];
      for (int l = 0; l < c; ++l) t = fma(-w.M[i + (int64_t)l * n], w.G[l + (int64_t)c * ldg], t);
      w.M[i + (int64_t)c * n] = t / w.G[c + (int64_t)c * ldg];
    }
  }
  __syncthreads();
  // ---- 3./4. Hessenberg form and real Schur form (T in M, Schur vectors
  //         in Z), in FP64 (schur_f64) ...
  double hnorm = 0.0;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) hnorm = fmax(hnorm, fabs(w.M[t]));
  hnorm = block_sum(hnorm, red);  // a bound on max |m_ij|, used for the scale and zero tests
  if (schur_f64) {
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) w.Z[t] = (t % (n + 1)) == 0 ? 1.0 : 0.0;
    __syncthreads();
    hessenberg_f64(w.M, w.Z, n, w.v, red, &sh_beta, &sh_tau);
    double hm = 0.0;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) hm = fmax(hm, fabs(w.M[t]));
    __shared__ double sh_hm[32];
    for (int o = 16; o > 0; o >>= 1) hm = fmax(hm, __shfl_xor_sync(0xffffffffu, hm, o));
    if ((threadIdx.x & 31) == 0) sh_hm[threadIdx.x >> 5] = hm;
    if (threadIdx.x == 0) {
      sh_u = n - 1;
      sh_iter = 0;
      sh_total = 0;
      sh_fail = 0;
    }
    __syncthreads();
    hm = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) hm = fmax(hm, sh_hm[q]);
    francis_f64(w.M, w.Z, n, w.wr, w.wi, hm, &sh_u, &sh_l, &sh_iter, &sh_total, &sh_fail);
    __syncthreads();
  } else {
  //         ... or in double-float. Both are long chains of small dependent steps, and on this
  //         GPU an FP64 instruction costs a warp ~64 cycles even with one
  //         lane active, so they run in double-float arithmetic on the FP32
  //         pipe (about 48 significant bits): M, scaled by a power of two
  //         (exact) so that its entries stay well inside the FP32 exponent
  //         range, is converted once into the F workspace (leading dimension
  //         n+1, conflict-free column sweeps), Z into the M workspace; the
  //         Schur-vector updates run on other warps than the row updates of
  //         H; T (scaled back), Z and the eigenvalues return to FP64.
  __shared__ double sh_scale;
  if (threadIdx.x == 0) {
    int ex = 0;
    if (hnorm > 0.0 && isfinite(hnorm)) frexp(hnorm, &ex);
    sh_scale = ldexp(1.0, -ex);
  }
  __syncthreads();
  const double hscale = sh_scale;
  const int ldh = n + 1;
  float2* Hd = reinterpret_cast<float2*>(w.F);
  float2* Zd = reinterpret_cast<float2*>(w.M);
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int r = t % n, c = t / n;
    Hd[r + (int64_t)c * ldh] = df_make(w.M[t] * hscale);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x)
    Zd[t] = make_float2((t % (n + 1)) == 0 ? 1.f : 0.f, 0.f);
  __syncthreads();
  hessenberg_df(Hd, ldh, Zd, n, reinterpret_cast<float2*>(w.v));
  __shared__ float sh_hmax;
  {
    float hm = 0.f;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) hm = fmaxf(hm, fabsf(Hd[t % n + (int64_t)(t / n) * ldh].x));
    for (int o = 16; o > 0; o >>= 1) hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, o));
    if (threadIdx.x == 0) sh_hmax = 0.f;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(&sh_hmax), __float_as_int(hm));
  }
  if (threadIdx.x == 0) {
    sh_u = n - 1;
    sh_iter = 0;
    sh_total = 0;
    sh_fail = 0;
  }
  __syncthreads();
  francis_df(Hd, ldh, Zd, n, w.wr, w.wi, sh_hmax, &sh_u, &sh_l, &sh_iter, &sh_total, &sh_fail);
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) w.Z[t] = df_to_double(Zd[t]);
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int r = t % n, c = t / n;
    w.M[t] = df_to_double(Hd[r + (int64_t)c * ldh]) / hscale;
  }
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    w.wr[t] /= hscale;
    w.wi[t] /= hscale;
  }
  }  // double-float Schur form
  double* H = w.M;
#define HH(i, j) H[(i) + (int64_t)(j) * n]
  __syncthreads();
  if (sh_fail) {
    if (threadIdx.x == 0) { *status_out = 2; *knew_out = 0; }
    return;
  }
  // ---- 5. selection: eigenvalues mu of largest modulus (theta = 1/mu smallest).
  //         |mu|^2 and Re theta = Re mu / |mu|^2 once per eigenvalue (in
  //         parallel, into X as scratch), then a serial pick of the best
  //         remaining entity; a complex pair is one entity (its first member,
  //         wi > 0) and is taken only if both fit. The scan compares integer
  //         images of the FP64 keys (a non-negative double orders like its
  //         bit pattern; a signed one like the pattern with the magnitude bits
  //         flipped when negative), which decide exactly as the FP64
  //         comparisons do but run on the integer pipe; the tie bounds
  //         |mu_best|^2 (1 +- 2e-12) are formed in FP64 when the best changes.
  double* mag2 = w.X;
  long long* rkey = reinterpret_cast<long long*>(w.X + n);
  int* used = w.sel + n + 1;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double m2 = w.wr[i] * w.wr[i] + w.wi[i] * w.wi[i];
    mag2[i] = m2;
    const double rt = m2 > 0.0 ? w.wr[i] / m2 : 0.0;
    const long long bits = __double_as_longlong(rt == 0.0 ? 0.0 : rt);
    rkey[i] = bits < 0 ? (bits ^ 0x7fffffffffffffffLL) : bits;
    used[i] = (w.wi[i] < 0.0 || !(m2 > 0.0)) ? 1 : 0;
  }
  // the scan's operands in shared memory (n <= kSelMax; else from X)
  constexpr int kSelMax = 256;
  __shared__ long long sel_m[kSelMax], sel_r[kSelMax];
  __shared__ int sel_u[kSelMax];
  const bool sel_sm = n <= kSelMax;
  __syncthreads();
  if (sel_sm)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      sel_m[i] = __double_as_longlong(mag2[i]);
      sel_r[i] = rkey[i];
      sel_u[i] = used[i];
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    int taken = 0, ns = 0;
    const double tie_hi = 1.0 + 2e-12, tie_lo = 1.0 - 2e-12;
    long long* km = sel_sm ? sel_m : nullptr;
    long long* kr = sel_sm ? sel_r : rkey;
    int* ku = sel_sm ? sel_u : used;
    while (taken < k) {
      int best = -1;
      long long bhi = 0, blo = 0, brk = 0;
      for (int i = 0; i < n; ++i) {
        if (ku[i]) continue;
        const long long m = km ? km[i] : __double_as_longlong(mag2[i]);  // mag2 > 0 here
        const long long rk = kr[i];
        if (best < 0 || m > bhi || (m >= blo && rk < brk)) {
          best = i;
          bhi = __double_as_longlong(mag2[i] * tie_hi);
          blo = __double_as_longlong(mag2[i] * tie_lo);
          brk = rk;
        }
      }
      if (best < 0) break;
      const int need = w.wi[best] > 0.0 ? 2 : 1;
      if (taken + need > k) break;
      ku[best] = 1;
      w.sel[ns++] = best;
      taken += need;
    }
    w.sel[ns] = -1;
    sh_knew = taken;
    sh_l = ns;
  }
  __syncthreads();
  const int knew = sh_knew;
  const int nsel = sh_l;
  if (knew == 0) {
    if (threadIdx.x == 0) { *status_out = 3; *knew_out = 0; }
    return;
  }
  // ---- 6. eigenvectors of T by back substitution (one thread per entity).
  for (int e = threadIdx.x; e < nsel; e += blockDim.x) {
    int col = 0;
    for (int t = 0; t < e; ++t) col += w.wi[w.sel[t]] > 0.0 ? 2 : 1;
    const int i = w.sel[e];
    double* xr = w.X + (int64_t)col * n;
    const double small = eps * (hnorm > 0.0 ? hnorm : 1.0);
    if (w.wi[i] == 0.0) {
      const double lam = H[i + (int64_t)i * n];
      for (int r = 0; r < n; ++r) xr[r] = 0.0;
      xr[i] = 1.0;
      int r = i - 1;
      while (r >= 0) {
        const bool blk = r > 0 && H[r + (int64_t)(r - 1) * n] != 0.0;
        if (!blk) {
          double s = 0.0;
          for (int c = r + 1; c <= i; ++c) s = fma(H[r + (int64_t)c * n], xr[c], s);
          double den = H[r + (int64_t)r * n] - lam;
          if (fabs(den) < small) den = small;
          xr[r] = -s / den;
          r -= 1;
        } else {
          double s1 = 0.0, s2 = 0.0;
          for (int c = r + 1; c <= i; ++c) {
            s1 = fma(H[(r - 1) + (int64_t)c * n], xr[c], s1);
            s2 = fma(H[r + (int64_t)c * n], xr[c], s2);
          }
          const double a = H[(r - 1) + (int64_t)(r - 1) * n] - lam, b = H[(r - 1) + (int64_t)r * n];
          const double c = H[r + (int64_t)(r - 1) * n], d = H[r + (int64_t)r * n] - lam;
          double det = a * d - b * c;
          if (fabs(det) < small * small) det = small * small;
          xr[r - 1] = (-s1 * d + b * s2) / det;
          xr[r] = (-a * s2 + c * s1) / det;
          r -= 2;
        }
      }
    } else {
      // complex pair at (i, i+1); eigenvalue lambda = wr + i*wi (wi > 0)
      double* xi = xr + n;
      const cplx lam = {w.wr[i], w.wi[i]};
      for (int r = 0; r < n; ++r) { xr[r] = 0.0; xi[r] = 0.0; }
      const double p = H[i + (int64_t)i * n], q = H[i + (int64_t)(i + 1) * n];
      const double rr = H[(i + 1) + (int64_t)i * n], ss = H[(i + 1) + (int64_t)(i + 1) * n];
      // null vector of [[p - lam, q], [rr, ss - lam]]
      if (fabs(q) >= fabs(rr)) {
        xr[i] = q; xi[i] = 0.0;
        xr[i + 1] = lam.re - p; xi[i + 1] = lam.im;
      } else {
        xr[i] = lam.re - ss; xi[i] = lam.im;
        xr[i + 1] = rr; xi[i + 1] = 0.0;
      }
      int r = i - 1;
      while (r >= 0) {
        const bool blk = r > 0 && H[r + (int64_t)(r - 1) * n] != 0.0;
        if (!blk) {
          cplx s = {0.0, 0.0};
          for (int c = r + 1; c <= i + 1; ++c) {
            s.re = fma(H[r + (int64_t)c * n], xr[c], s.re);
            s.im = fma(H[r + (int64_t)c * n], xi[c], s.im);
          }
          cplx den = {H[r + (int64_t)r * n] - lam.re, -lam.im};
          if (fabs(den.re) + fabs(den.im) < small) den.re = small;
          const cplx val = cdiv({-s.re, -s.im}, den);
          xr[r] = val.re;
          xi[r] = val.im;
          r -= 1;
        } else {
          cplx s1 = {0.0, 0.0}, s2 = {0.0, 0.0};
          for (int c = r + 1; c <= i + 1; ++c) {
            s1.re = fma(H[(r - 1) + (int64_t)c * n], xr[c], s1.re);
            s1.im = fma(H[(r - 1) + (int64_t)c * n], xi[c], s1.im);
            s2.re = fma(H[r + (int64_t)c * n], xr[c], s2.re);
            s2.im = fma(H[r + (int64_t)c * n], xi[c], s2.im);
          }
          const cplx a = {H[(r - 1) + (int64_t)(r - 1) * n] - lam.re, -lam.im};
          const cplx b = {H[(r - 1) + (int64_t)r * n], 0.0};
          const cplx c = {H[r + (int64_t)(r - 1) * n], 0.0};
          const cplx d = {H[r + (int64_t)r * n] - lam.re, -lam.im};
          cplx det = cmul(a, d);
          const cplx bc = cmul(b, c);
          det.re -= bc.re;
          det.im -= bc.im;
          if (fabs(det.re) + fabs(det.im) < small * small) det.re = small * small;
          const cplx ms1 = {-s1.re, -s1.im}, ms2 = {-s2.re, -s2.im};
          cplx t1 = cmul(ms1, d), t2 = cmul(b, ms2);
          const cplx x1 = cdiv({t1.re - t2.re, t1.im - t2.im}, det);
          t1 = cmul(a, ms2);
          t2 = cmul(c, ms1);
          const cplx x2 = cdiv({t1.re - t2.re, t1.im - t2.im}, det);
          xr[r - 1] = x1.re; xi[r - 1] = x1.im;
          xr[r] = x2.re; xi[r] = x2.im;
          r -= 2;
        }
      }
    }
  }
  __syncthreads();
  // ---- 7. back to M'' coordinates: Y = Z X (stored in F, ld n), then
  //         orthonormalise the columns (two Gram-Schmidt passes) into X.
  double* Y = w.F;
  for (int t = threadIdx.x; t < n * knew; t += blockDim.x) {
    const int r = t % n, c = t / n;
    double s = 0.0;
    for (int l2 = 0; l2 < n; ++l2) s = fma(w.Z[r + (int64_t)l2 * n], w.X[l2 + (int64_t)c * n], s);
    Y[t] = s;
  }
  __syncthreads();
  // classical Gram-Schmidt, two passes: per pass all inner products with
  // the kept columns at once (a warp per inner product), then one update
  double* sh_d = w.v;  // the inner products (kept <= n of them; v is free here)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  int kept = 0;
  for (int c = 0; c < knew; ++c) {
    double* yc = Y + (int64_t)c * n;
    double s0 = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) s0 = fma(yc[r], yc[r], s0);
    const double n0 = sqrt(block_sum(s0, red));
    for (int pass = 0; pass < 2 && kept > 0; ++pass) {
      for (int c2 = warp; c2 < kept; c2 += nwarp) {
        const double* qc = w.X + (int64_t)c2 * n;
        double d = 0.0;
        for (int r = lane; r < n; r += 32) d = fma(qc[r], yc[r], d);
        d = warp_sum(d);
        if (lane == 0) sh_d[c2] = d;
      }
      __syncthreads();
      for (int r = threadIdx.x; r < n; r += blockDim.x) {
        double t = yc[r];
        for (int c2 = 0; c2 < kept; ++c2) t = fma(-sh_d[c2], w.X[r + (int64_t)c2 * n], t);
        yc[r] = t;
      }
      __syncthreads();
    }
    double s1 = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) s1 = fma(yc[r], yc[r], s1);
    const double n1 = sqrt(block_sum(s1, red));
    __syncthreads();
    if (n1 > 1e-10 * n0 && n1 > 0.0) {
      double* qk = w.X + (int64_t)kept * n;
      for (int r = threadIdx.x; r < n; r += blockDim.x) qk[r] = yc[r] / n1;
      ++kept;
    }
    __syncthreads();
  }
  // ---- 8. QC = Q_G [Q2; 0] ((n+1) x kept), PU = R_G^{-1} Q2 (n x kept).
  for (int t = threadIdx.x; t < (n + 1) * kept; t += blockDim.x) {
    const int r = t % (n + 1), c = t / (n + 1);
    QC[r + (int64_t)c * ldqc] = r < n ? w.X[r + (int64_t)c * n] : 0.0;
  }
  __syncthreads();
  // Q_G applied to each column by a warp (lanes over rows): the columns are
  // independent, so no block barrier between reflectors
  // (two columns per warp at a time, so the two dependent chains overlap)
  for (int j0 = 2 * warp; j0 < kept; j0 += 2 * nwarp) {
    const bool two = j0 + 1 < kept;
    double* colA = QC + (int64_t)j0 * ldqc;
    double* colB = QC + (int64_t)(two ? j0 + 1 : j0) * ldqc;
    for (int c = n - 1; c >= 0; --c) {
      const int len = n + 1 - c;
      const double* vv = w.G + (int64_t)c * ldg + c;  // vv[0] holds R_G(c,c); the reflector has v[0] = 1
      double sa = 0.0, sb = 0.0;
      for (int i = lane; i < len; i += 32) {
        const double vi = i == 0 ? 1.0 : vv[i];
        sa = fma(vi, colA[c + i], sa);
        sb = fma(vi, colB[c + i], sb);
      }
      const double tc = w.tau[c];
      sa = warp_sum(sa) * tc;
      sb = warp_sum(sb) * tc;
      for (int i = lane; i < len; i += 32) {
        const double vi = i == 0 ? 1.0 : vv[i];
        colA[c + i] = fma(-sa, vi, colA[c + i]);
        if (two) colB[c + i] = fma(-sb, vi, colB[c + i]);
      }
      __syncwarp();
    }
  }
  // PU = R_G^{-1} Q2 by column-oriented back substitution, a warp per
  // column: pu_r = t_r / R_rr, then t_i -= R_ir pu_r for i < r (lanes)
  double* rdiag = w.v;  // 1 / R_G(r, r)
  for (int r = threadIdx.x; r < n; r += blockDim.x) rdiag[r] = 1.0 / w.G[r + (int64_t)r * ldg];
  __syncthreads();
  for (int j = warp; j < kept; j += nwarp) {
    double* pu = PU + (int64_t)j * ldpu;
    for (int r = lane; r < n; r += 32) pu[r] = w.X[r + (int64_t)j * n];
    __syncwarp();
    for (int r = n - 1; r >= 0; --r) {
      const double pr = pu[r] * rdiag[r];
      __syncwarp();
      if (lane == 0) pu[r] = pr;
      for (int i = lane; i < r; i += 32) pu[i] = fma(-w.G[i + (int64_t)r * ldg], pr, pu[i]);
      __syncwarp();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *knew_out = kept;
    *status_out = 0;
  }
#undef HH
}

// Solver wrapper: builds G and F from the cycle's B, H and Gram, runs the
// core, folds the column scales of the stored V into QC and PU.
__global__ void __launch_bounds__(kHRThreads) k_harmonic_ritz(SolveState* s, SmallBuffers b, int kc, int jj, int k,
                                                              int use_smem, int schur_f64) {
  extern __shared__ double dsm[];
  const int n = kc + jj;
  double* base = use_smem ? dsm : b.hrws;
  HRWork w = hr_carve(base, n);
  const int ldg = n + 1;
  const int ldh = b.m + 1;
  for (int t = threadIdx.x; t < (n + 1) * n; t += blockDim.x) {
    const int r = t % (n + 1), c = t / (n + 1);
    double gv = 0.0, fv = 0.0;
    if (r < kc && c < kc) {
      gv = r == c ? 1.0 : 0.0;
      fv = b.gram[r + (int64_t)c * (kc + jj + 1)];
    } else if (r < kc) {
      gv = b.B[r + (int64_t)(c - kc) * b.kmax];
    } else if (c < kc) {
      fv = b.sv[r - kc] * b.gram[r + (int64_t)c * (kc + jj + 1)];
    } else {
      gv = b.H[(r - kc) + (int64_t)(c - kc) * ldh];
      fv = (r - kc) == (c - kc) ? 1.0 : 0.0;
    }
    w.G[r + (int64_t)c * ldg] = gv;
    w.F[r + (int64_t)c * ldg] = fv;
  }
  __syncthreads();
  __shared__ int knew, st;
  hr_core(w, n, k, b.QC, n + 1, b.PU, n, &knew, &st, schur_f64);
  __syncthreads();
  // fold the stored-column scales (v_l = sv[l] q_l) into the coefficients
  for (int t = threadIdx.x; t < (n + 1) * knew; t += blockDim.x) {
    const int r = t % (n + 1), c = t / (n + 1);
    if (r >= kc) b.QC[r + (int64_t)c * (n + 1)] *= b.sv[r - kc];
  }
  for (int t = threadIdx.x; t < n * knew; t += blockDim.x) {
    const int r = t % n, c = t / n;
    if (r >= kc) b.PU[r + (int64_t)c * n] *= b.sv[r - kc];
  }
  if (threadIdx.x == 0) {
    s->knew = st == 0 ? knew : kc;
    s->hr_status = st;
  }
}

__global__ void __launch_bounds__(kHRThreads) k_harmonic_ritz_small(int n, const double* G, const double* F, int k,
                                                                    double* QC, double* PU, int* knew_out,
                                                                    double* ws, int use_smem, int schur_f64) {
  extern __shared__ double dsm[];
  double* base = use_smem ? dsm : ws;
  HRWork w = hr_carve(base, n);
  for (int t = threadIdx.x; t < (n + 1) * n; t += blockDim.x) {
    w.G[t] = G[t];
    w.F[t] = F[t];
  }
  __syncthreads();
  __shared__ int knew, st;
  hr_core(w, n, k, QC, n + 1, PU, n, &knew, &st, schur_f64);
  __syncthreads();
  if (threadIdx.x == 0) *knew_out = st == 0 ? knew : -st;
}

// Cholesky G = R^T R of a k x k Gram matrix and R^{-1} (upper), one thread;
// used by the CholQR that forms C from U (C~ = A U = C R). status: 0 ok, 1 not SPD.
__global__ void k_chol_rinv(int k, const double* G, double* Rinv, double* Rw, int* status) {
  if (threadIdx.x != 0) return;
  for (int t = 0; t < k * k; ++t) Rw[t] = 0.0;
  for (int j = 0; j < k; ++j) {
    double d = G[j + j * k];
    for (int l = 0; l < j; ++l) d -= Rw[l + j * k] * Rw[l + j * k];
    if (!(d > 0.0)) {
      *status = 1;
      return;
    }
    const double rjj = sqrt(d);
    Rw[j + j * k] = rjj;
    for (int c = j + 1; c < k; ++c) {
      double t = G[j + c * k];
      for (int l = 0; l < j; ++l) t -= Rw[l + j * k] * Rw[l + c * k];
      Rw[j + c * k] = t / rjj;
    }
  }
  // Rinv = R^{-1}: solve R X = I column by column (X upper triangular)
  for (int c = 0; c < k; ++c) {
    for (int r = k - 1; r >= 0; --r) {
      double t = r == c ? 1.0 : 0.0;
      for (int l = r + 1; l <= c; ++l) t -= Rw[r + l * k] * Rinv[l + c * k];
      Rinv[r + c * k] = r > c ? 0.0 : t / Rw[r + r * k];
    }
  }
  *status = 0;
}

// Start of an Arnoldi cycle: g = rho e_1, v_1 = r / rho (stored normalised in
// column 0), no steps taken.
__global__ void k_cycle_init(SolveState* s, SmallBuffers b) {
  const double rho = sqrt(s->rho2);
  for (int i = threadIdx.x; i <= b.m; i += blockDim.x) b.g[i] = i == 0 ? rho : 0.0;
  if (threadIdx.x == 0) {
    b.sv[0] = 1.0;  // column 0 holds p_0 = r / rho
    s->done = rho > 0.0 ? 0 : 1;
    s->jj = 0;
    s->nspmv = 0;
    s->upd_mode = 2;
    s->scal[3] = 1.0;
  }
}

// ||b|| from the reduced sum of squares and the absolute tolerance.
__global__ void k_set_tol(SolveState* s, double tol) {
  if (threadIdx.x != 0) return;
  s->bnorm = sqrt(s->nrm2[0]);
  s->tolabs = tol * s->bnorm;
}

__global__ void k_set_tolabs(SolveState* s, double tolabs) {
  if (threadIdx.x == 0) s->tolabs = tolabs;
}

__global__ void k_set_scalar(SolveState* s, int which) {
  if (threadIdx.x != 0) return;
  if (which == 0) s->done = 0;
}

size_t hr_doubles_host(int n) { return (size_t)2 * (n + 1) * n + (size_t)3 * n * n + 6 * (size_t)n + 8; }

}  // namespace

size_t harmonic_ritz_ws_doubles(int n) { return hr_doubles_host(n); }

cudaError_t launch_dcgs_coef(SolveState* s, SmallBuffers b, int kc, int j, int final_pass, cudaStream_t st) {
  k_dcgs_coef<<<1, 128, (3 * (size_t)b.m + 2) * sizeof(double), st>>>(s, b, kc, j, final_pass);
  return cudaGetLastError();
}

cudaError_t launch_cycle_solve(SolveState* s, SmallBuffers b, int kc, cudaStream_t st) {
  if (b.m <= kSolveStageMax) {
    const size_t smem = ((size_t)b.m * b.m + 3 * (size_t)b.m) * sizeof(double);
    k_cycle_solve<true><<<1, kSolveThreads, smem, st>>>(s, b, kc);
  } else {
    k_cycle_solve<false><<<1, kSolveThreads, 3 * (size_t)b.m * sizeof(double), st>>>(s, b, kc);
  }
  return cudaGetLastError();
}

static constexpr size_t kHRSmemMax = 200 * 1024;

cudaError_t launch_harmonic_ritz(SolveState* s, SmallBuffers b, int kc, int jj, int k, bool schur_f64,
                                 cudaStream_t st) {
  const int n = kc + jj;
  const size_t bytes = hr_doubles_host(n) * sizeof(double);
  const int use_smem = bytes <= kHRSmemMax ? 1 : 0;
  // one-time attribute setup per device
  static std::atomic<uint64_t> done{0};
  once_per_device(done, [] {
    cudaFuncSetAttribute(k_harmonic_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHRSmemMax);
  });
  k_harmonic_ritz<<<1, kHRThreads, use_smem ? bytes : 0, st>>>(s, b, kc, jj, k, use_smem, schur_f64 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_harmonic_ritz_small(int n, const double* G, const double* F, int k, double* QC, double* PU,
                                       int* knew, double* ws, bool schur_f64, cudaStream_t st) {
  const size_t bytes = hr_doubles_host(n) * sizeof(double);
  const int use_smem = bytes <= kHRSmemMax ? 1 : 0;
  // one-time attribute setup per device
  static std::atomic<uint64_t> done{0};
  once_per_device(done, [] {
    cudaFuncSetAttribute(k_harmonic_ritz_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHRSmemMax);
  });
  k_harmonic_ritz_small<<<1, kHRThreads, use_smem ? bytes : 0, st>>>(n, G, F, k, QC, PU, knew, ws, use_smem,
                                                                     schur_f64 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_chol_rinv(int k, const double* G, double* Rinv, double* Rw, int* status, cudaStream_t st) {
  k_chol_rinv<<<1, 32, 0, st>>>(k, G, Rinv, Rw, status);
  return cudaGetLastError();
}

cudaError_t launch_cycle_init(SolveState* s, SmallBuffers b, cudaStream_t st) {
  k_cycle_init<<<1, 128, 0, st>>>(s, b);
  return cudaGetLastError();
}

cudaError_t launch_set_tol(SolveState* s, double tol, cudaStream_t st) {
  k_set_tol<<<1, 32, 0, st>>>(s, tol);
  return cudaGetLastError();
}

cudaError_t launch_set_tolabs(SolveState* s, double tolabs, cudaStream_t st) {
  k_set_tolabs<<<1, 32, 0, st>>>(s, tolabs);
  return cudaGetLastError();
}

cudaError_t launch_set_scalar(SolveState* s, int which, cudaStream_t st) {
  k_set_scalar<<<1, 32, 0, st>>>(s, which);
  return cudaGetLastError();
}

}  // namespace rk
