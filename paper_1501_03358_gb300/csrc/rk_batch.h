// Batched rBiCGStab phase (the batched workload's second hybrid phase): one
// launch per iteration phase serves every problem of a batch. Internal to
// librk.
//
// A launch walks a work list of (problem, block) items with a persistent
// grid (any grid size); item (i, b) does exactly what block b of the
// single-problem kernel does for problem i (the same device code, the same
// element partition by that problem's own block count, the same partial
// sums and the same last-block reduction through that problem's own
// counter), so a batched solve gives bit for bit the result of the solve
// alone, whatever the grid size the tuner picks.
#pragma once
#include "rk_internal.h"
#include "rk_bicg.h"

namespace rk {

struct BatchProb {
  Dims d;
  int S;           // 7 or 19
  int kc;          // recycle dimension (FP64 columns of C)
  int nblk;        // red_blocks(n): blocks of the single-problem streaming kernels
  int f32;         // 1: the FP32 operator of RK_MIXED, 0: FP64
  int gx, gy, gz, zchunk;  // the single-problem stencil grid
  int64_t ld;
  const double* coef;
  const double* dinv;
  const float* coef32;
  const float* dinv32;
  BicgVecs v;
  BicgScalars* bs;
  const double* C;
  double* eta1;
  double* eta2;
  double* xi;
  double* part;
  unsigned* counter;
};

// work-list items: x = problem index, y = block (streaming kernels) or tile
// index (stencil: bx + gx (by + gy bz))
cudaError_t launch_batch_bicg_p(const BatchProb* P, const int2* items, int nitems, int grid, cudaStream_t st);
cudaError_t launch_batch_bicg_alpha(const BatchProb* P, int nprob, cudaStream_t st);
cudaError_t launch_batch_bicg_s(const BatchProb* P, const int2* items, int nitems, int grid, cudaStream_t st);
cudaError_t launch_batch_bicg_t(const BatchProb* P, const int2* items, int nitems, int grid, cudaStream_t st);
cudaError_t launch_batch_bicg_r(const BatchProb* P, const int2* items, int nitems, int grid, cudaStream_t st);
// which = 0: [C^T v, r~^T v] -> eta1; 1: C^T t -> eta2 (problems with kc > 0)
cudaError_t launch_batch_dots(const BatchProb* P, const int2* items, int nitems, int which, int grid,
                              cudaStream_t st);
// which = 0: v = A M^{-1} p; 1: t = A M^{-1} s (right point Jacobi; FP64 or
// FP32 operator per problem); all problems of one launch have S bands
cudaError_t launch_batch_stencil(const BatchProb* P, const int2* tiles, int ntiles, int S, int which, int grid,
                                 cudaStream_t st);

}  // namespace rk
