/*
 * Oracle (test infrastructure only; never linked into the product library).
 *
 * Plain C loops for the banded structured-grid operator of Sec. 2.1 ("Data
 * Layout": 7 or 19 coefficients per cell in diagonal storage) and the right
 * point-Jacobi preconditioner (Sec. 2.1, "Preconditioners"; applied from the
 * right as for BiCGStab).
 *
 * Every output element is evaluated in a fixed order:
 *   z_q   = v_q * dinv_q              (dinv_q = 1 / a_qq, IEEE divide)
 *   w_p   = coef[0][p] * z_p
 *   w_p   = fma(coef[s][p], z_nb(p,s), w_p)   for s = 1 .. S-1
 * Bands that point out of a non-periodic face are skipped (their
 * coefficients are zero by construction). Periodic axes wrap.
 *
 * Layout: coef is S contiguous bands of N = nx*ny*nz doubles, cell index
 * i + nx*(j + ny*k). Band offsets (dx,dy,dz):
 *   0 (0,0,0); 1 (-1,0,0) 2 (1,0,0) 3 (0,-1,0) 4 (0,1,0) 5 (0,0,-1) 6 (0,0,1);
 *   7 (-1,-1,0) 8 (1,-1,0) 9 (-1,1,0) 10 (1,1,0);
 *   11 (-1,0,-1) 12 (1,0,-1) 13 (-1,0,1) 14 (1,0,1);
 *   15 (0,-1,-1) 16 (0,1,-1) 17 (0,-1,1) 18 (0,1,1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static const int OFF[19][3] = {
    {0, 0, 0},
    {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1},
    {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0},
    {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1}, {1, 0, 1},
    {0, -1, -1}, {0, 1, -1}, {0, -1, 1}, {0, 1, 1},
};

/* neighbour coordinate along one axis; -1 when outside a non-periodic axis */
static int64_t wrap(int64_t c, int64_t n, int periodic) {
  if (c >= 0 && c < n) return c;
  if (!periodic) return -1;
  return c < 0 ? c + n : c - n;
}

/* y = A * (scale .* v); scale == NULL means the identity */
static void apply_core(int64_t nx, int64_t ny, int64_t nz, const uint8_t* per, int S,
                       const double* coef, const double* scale, const double* v, double* y) {
  const int64_t N = nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nz; ++k) {
    for (int64_t j = 0; j < ny; ++j) {
      for (int64_t i = 0; i < nx; ++i) {
        const int64_t p = i + nx * (j + ny * k);
        double zp = scale ? v[p] * scale[p] : v[p];
        double w = coef[p] * zp;
        for (int s = 1; s < S; ++s) {
          int64_t ii = wrap(i + OFF[s][0], nx, per[0]);
          int64_t jj = wrap(j + OFF[s][1], ny, per[1]);
          int64_t kk = wrap(k + OFF[s][2], nz, per[2]);
          if (ii < 0 || jj < 0 || kk < 0) continue;
          const int64_t q = ii + nx * (jj + ny * kk);
          double zq = scale ? v[q] * scale[q] : v[q];
          w = fma(coef[(int64_t)s * N + p], zq, w);
        }
        y[p] = w;
      }
    }
  }
}

/* dinv[p] = 1 / coef[0][p] */
void oracle_jacobi_inverse(int64_t n, const double* coef, double* dinv) {
  for (int64_t p = 0; p < n; ++p) dinv[p] = 1.0 / coef[p];
}

/* w = A * M^{-1} v  (right point-Jacobi) */
void oracle_apply_prec(int64_t nx, int64_t ny, int64_t nz, const uint8_t* per, int S,
                       const double* coef, const double* dinv, const double* v, double* w) {
  apply_core(nx, ny, nz, per, S, coef, dinv, v, w);
}

/* w = A v */
void oracle_apply(int64_t nx, int64_t ny, int64_t nz, const uint8_t* per, int S,
                  const double* coef, const double* v, double* w) {
  apply_core(nx, ny, nz, per, S, coef, 0, v, w);
}

/* Mixed-precision inner operator (FP32): with c32 = RN32(coef), d32 =
 * RN32(1/a_pp) and z_q = RN32(RN32(v_q) * d32_q), w_p = RN32(c32_0 z_p) then
 * w_p = fmaf(c32_s, z_nb, w_p) in band order; the result widened to double. */
void oracle_apply_prec_f32(int64_t nx, int64_t ny, int64_t nz, const uint8_t* per, int S,
                           const double* coef, const double* dinv, const double* v, double* y) {
  const int64_t N = nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nz; ++k) {
    for (int64_t j = 0; j < ny; ++j) {
      for (int64_t i = 0; i < nx; ++i) {
        const int64_t p = i + nx * (j + ny * k);
        float zp = (float)v[p] * (float)dinv[p];
        float w = (float)coef[p] * zp;
        for (int s = 1; s < S; ++s) {
          int64_t ii = wrap(i + OFF[s][0], nx, per[0]);
          int64_t jj = wrap(j + OFF[s][1], ny, per[1]);
          int64_t kk = wrap(k + OFF[s][2], nz, per[2]);
          if (ii < 0 || jj < 0 || kk < 0) continue;
          const int64_t q = ii + nx * (jj + ny * kk);
          float zq = (float)v[q] * (float)dinv[q];
          w = fmaf((float)coef[(int64_t)s * N + p], zq, w);
        }
        y[p] = (double)w;
      }
    }
  }
}

/* r = b - A x, element by element: r_p = b_p - (A x)_p */
void oracle_residual(int64_t nx, int64_t ny, int64_t nz, const uint8_t* per, int S,
                     const double* coef, const double* b, const double* x, double* r) {
  const int64_t N = nx * ny * nz;
  apply_core(nx, ny, nz, per, S, coef, 0, x, r);
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < N; ++p) r[p] = b[p] - r[p];
}

/*
 * The "Jacobi preconditioner" of Sec. 2.1 (reading of this implementation):
 * overlapping sub-domains solved inexactly by damped Jacobi, then one damped
 * point-Jacobi sweep on the global problem. z = M^{-1} r:
 *   - the grid is cut into boxes of bx x by x bz owned cells (the last box
 *     along an axis may be smaller); each box is extended by `ov` cells on
 *     every side (wrapping on periodic axes; cells beyond a non-periodic face
 *     are absent). The extended cells are the local unknowns (a cell reached
 *     twice by wrapping is two unknowns);
 *   - local problem: A restricted to the extended cells (couplings to cells
 *     outside the extended box dropped); `sweeps` damped Jacobi sweeps from
 *     zero, each  s = c_0 z_e, s = fma(c_s, z_nb, s) in band order over the
 *     present neighbours, t = r_e - s, u = dinv_e * t, z_e <- fma(omega, u, z_e);
 *   - restriction: every cell takes the value of its own box's local solve;
 *   - one global sweep of the same form with the full operator:
 *     z_p <- fma(omega, dinv_p * (r_p - (A z)_p), z_p).
 */
void oracle_schwarz_jacobi(int64_t nx, int64_t ny, int64_t nz, const uint8_t* per, int S,
                           const double* coef, const double* dinv, int bx, int by, int bz, int ov,
                           int sweeps, double omega, const double* r, double* z) {
  const int64_t N = nx * ny * nz;
  const int64_t nbx = (nx + bx - 1) / bx, nby = (ny + by - 1) / by, nbz = (nz + bz - 1) / bz;
#pragma omp parallel for schedule(dynamic)
  for (int64_t box = 0; box < nbx * nby * nbz; ++box) {
    const int64_t ib = box % nbx, jb = (box / nbx) % nby, kb = box / (nbx * nby);
    const int64_t x0 = ib * bx, y0 = jb * by, z0 = kb * bz;
    const int64_t x1 = x0 + bx < nx ? x0 + bx : nx, y1 = y0 + by < ny ? y0 + by : ny, z1 = z0 + bz < nz ? z0 + bz : nz;
    const int64_t ex = (x1 - x0) + 2 * ov, ey = (y1 - y0) + 2 * ov, ez = (z1 - z0) + 2 * ov;
    const int64_t ne = ex * ey * ez;
    int64_t* gidx = (int64_t*)malloc(sizeof(int64_t) * ne);
    double* za = (double*)calloc(ne, sizeof(double));
    double* zb = (double*)calloc(ne, sizeof(double));
    for (int64_t c = 0; c < ez; ++c)
      for (int64_t b = 0; b < ey; ++b)
        for (int64_t a = 0; a < ex; ++a) {
          const int64_t gi = wrap(x0 - ov + a, nx, per[0]), gj = wrap(y0 - ov + b, ny, per[1]),
                        gk = wrap(z0 - ov + c, nz, per[2]);
          gidx[a + ex * (b + ey * c)] = (gi < 0 || gj < 0 || gk < 0) ? -1 : gi + nx * (gj + ny * gk);
        }
    for (int sw = 0; sw < sweeps; ++sw) {
      for (int64_t c = 0; c < ez; ++c)
        for (int64_t b = 0; b < ey; ++b)
          for (int64_t a = 0; a < ex; ++a) {
            const int64_t e = a + ex * (b + ey * c);
            const int64_t p = gidx[e];
            if (p < 0) continue;
            double s = coef[p] * za[e];
            for (int t = 1; t < S; ++t) {
              const int64_t aa = a + OFF[t][0], bb = b + OFF[t][1], cc = c + OFF[t][2];
              if (aa < 0 || aa >= ex || bb < 0 || bb >= ey || cc < 0 || cc >= ez) continue;
              const int64_t q = aa + ex * (bb + ey * cc);
              if (gidx[q] < 0) continue;
              s = fma(coef[(int64_t)t * N + p], za[q], s);
            }
            const double u = dinv[p] * (r[p] - s);
            zb[e] = fma(omega, u, za[e]);
          }
      double* tmp = za;
      za = zb;
      zb = tmp;
    }
    for (int64_t k = z0; k < z1; ++k)
      for (int64_t j = y0; j < y1; ++j)
        for (int64_t i = x0; i < x1; ++i)
          z[i + nx * (j + ny * k)] = za[(i - x0 + ov) + ex * ((j - y0 + ov) + ey * (k - z0 + ov))];
    free(gidx);
    free(za);
    free(zb);
  }
  /* the global point-Jacobi sweep */
  double* az = (double*)malloc(sizeof(double) * N);
  apply_core(nx, ny, nz, per, S, coef, 0, z, az);
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < N; ++p) {
    const double u = dinv[p] * (r[p] - az[p]);
    az[p] = fma(omega, u, z[p]);
  }
  for (int64_t p = 0; p < N; ++p) z[p] = az[p];
  free(az);
}

/*
 * FP32 restatements for the mixed precision (RK_MIXED) of the library, each
 * the FP64 procedure above with every operand rounded to FP32 once (bands
 * c32 = RN32(coef), d32 = RN32(1/a_pp), the input vector, omega) and every
 * operation one FP32 rounding, in the same order.
 *
 * mode 1: w = A32 v32 (w_p = RN32(c32_0 v_p), then fmaf in band order);
 * mode 3: w = d32 .* (A32 v32) (the product, then one rounded multiplication).
 */
void oracle_apply_f32(int64_t nx, int64_t ny, int64_t nz, const uint8_t* per, int S, const double* coef,
                      const double* dinv, int mode, const double* v, double* y) {
  const int64_t N = nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nz; ++k) {
    for (int64_t j = 0; j < ny; ++j) {
      for (int64_t i = 0; i < nx; ++i) {
        const int64_t p = i + nx * (j + ny * k);
        float w = (float)coef[p] * (float)v[p];
        for (int s = 1; s < S; ++s) {
          int64_t ii = wrap(i + OFF[s][0], nx, per[0]);
          int64_t jj = wrap(j + OFF[s][1], ny, per[1]);
          int64_t kk = wrap(k + OFF[s][2], nz, per[2]);
          if (ii < 0 || jj < 0 || kk < 0) continue;
          const int64_t q = ii + nx * (jj + ny * kk);
          w = fmaf((float)coef[(int64_t)s * N + p], (float)v[q], w);
        }
        if (mode == 3) w = w * (float)dinv[p];
        y[p] = (double)w;
      }
    }
  }
}

/*
 * The sub-domain preconditioner of oracle_schwarz_jacobi in FP32 (the
 * RK_MIXED variant): the same boxes, overlap, local damped Jacobi sweeps
 * from zero and restriction, then the global damped sweep
 *   y_p = fmaf(om32, d32_p * (r32_p - (A32 z)_p), z_p),
 * with r32 = RN32(r); the result widened to double.
 */
void oracle_schwarz_jacobi_f32(int64_t nx, int64_t ny, int64_t nz, const uint8_t* per, int S,
                               const double* coef, const double* dinv, int bx, int by, int bz, int ov,
                               int sweeps, double omega, const double* r, double* z) {
  const int64_t N = nx * ny * nz;
  const float om = (float)omega;
  const int64_t nbx = (nx + bx - 1) / bx, nby = (ny + by - 1) / by, nbz = (nz + bz - 1) / bz;
  float* zl = (float*)malloc(sizeof(float) * N);
#pragma omp parallel for schedule(dynamic)
  for (int64_t box = 0; box < nbx * nby * nbz; ++box) {
    const int64_t ib = box % nbx, jb = (box / nbx) % nby, kb = box / (nbx * nby);
    const int64_t x0 = ib * bx, y0 = jb * by, z0 = kb * bz;
    const int64_t x1 = x0 + bx < nx ? x0 + bx : nx, y1 = y0 + by < ny ? y0 + by : ny, z1 = z0 + bz < nz ? z0 + bz : nz;
    const int64_t ex = (x1 - x0) + 2 * ov, ey = (y1 - y0) + 2 * ov, ez = (z1 - z0) + 2 * ov;
    const int64_t ne = ex * ey * ez;
    int64_t* gidx = (int64_t*)malloc(sizeof(int64_t) * ne);
    float* za = (float*)calloc(ne, sizeof(float));
    float* zb = (float*)calloc(ne, sizeof(float));
    for (int64_t c = 0; c < ez; ++c)
      for (int64_t b = 0; b < ey; ++b)
        for (int64_t a = 0; a < ex; ++a) {
          const int64_t gi = wrap(x0 - ov + a, nx, per[0]), gj = wrap(y0 - ov + b, ny, per[1]),
                        gk = wrap(z0 - ov + c, nz, per[2]);
          gidx[a + ex * (b + ey * c)] = (gi < 0 || gj < 0 || gk < 0) ? -1 : gi + nx * (gj + ny * gk);
        }
    for (int sw = 0; sw < sweeps; ++sw) {
      for (int64_t c = 0; c < ez; ++c)
        for (int64_t b = 0; b < ey; ++b)
          for (int64_t a = 0; a < ex; ++a) {
            const int64_t e = a + ex * (b + ey * c);
            const int64_t p = gidx[e];
            if (p < 0) continue;
            float s = (float)coef[p] * za[e];
            for (int t = 1; t < S; ++t) {
              const int64_t aa = a + OFF[t][0], bb = b + OFF[t][1], cc = c + OFF[t][2];
              if (aa < 0 || aa >= ex || bb < 0 || bb >= ey || cc < 0 || cc >= ez) continue;
              const int64_t q = aa + ex * (bb + ey * cc);
              if (gidx[q] < 0) continue;
              s = fmaf((float)coef[(int64_t)t * N + p], za[q], s);
            }
            const float u = (float)dinv[p] * ((float)r[p] - s);
            zb[e] = fmaf(om, u, za[e]);
          }
      float* tmp = za;
      za = zb;
      zb = tmp;
    }
    for (int64_t k = z0; k < z1; ++k)
      for (int64_t j = y0; j < y1; ++j)
        for (int64_t i = x0; i < x1; ++i)
          zl[i + nx * (j + ny * k)] = za[(i - x0 + ov) + ex * ((j - y0 + ov) + ey * (k - z0 + ov))];
    free(gidx);
    free(za);
    free(zb);
  }
  /* the global sweep in FP32 */
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nz; ++k) {
    for (int64_t j = 0; j < ny; ++j) {
      for (int64_t i = 0; i < nx; ++i) {
        const int64_t p = i + nx * (j + ny * k);
        float w = (float)coef[p] * zl[p];
        for (int s = 1; s < S; ++s) {
          int64_t ii = wrap(i + OFF[s][0], nx, per[0]);
          int64_t jj = wrap(j + OFF[s][1], ny, per[1]);
          int64_t kk = wrap(k + OFF[s][2], nz, per[2]);
          if (ii < 0 || jj < 0 || kk < 0) continue;
          const int64_t q = ii + nx * (jj + ny * kk);
          w = fmaf((float)coef[(int64_t)s * N + p], zl[q], w);
        }
        const float u = ((float)r[p] - w) * (float)dinv[p];
        z[p] = (double)fmaf(om, u, zl[p]);
      }
    }
  }
  free(zl);
}
