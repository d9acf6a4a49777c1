// Device helpers shared by the streaming kernels: fixed-order (deterministic)
// warp/block reductions and the "last block finishes the grid reduction"
// pattern. Every sum here has an order fixed by the launch shape alone.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace rk {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block (blockDim.x a multiple of 32, <= 1024); result valid in
// every thread. `red` needs 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = lane < nw ? red[lane] : 0.0;
  t = warp_sum(t);
  return t;
}

// After a block has written its partials: returns true in every thread of
// the last block to arrive (which then owns the final reduction) and resets
// the counter for the next launch.
__device__ __forceinline__ bool arrive_last(unsigned* counter, int* flag_smem) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    *flag_smem = (t == gridDim.x * gridDim.y * gridDim.z - 1) ? 1 : 0;
  }
  __syncthreads();
  bool last = *flag_smem != 0;
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return last;
}

// The same for a reduction over nblocks blocks that need not be the whole
// grid (the batched launches, where one launch serves many problems).
__device__ __forceinline__ bool arrive_last_n(unsigned* counter, int* flag_smem, int nblocks) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    *flag_smem = (t == (unsigned)nblocks - 1u) ? 1 : 0;
  }
  __syncthreads();
  bool last = *flag_smem != 0;
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return last;
}

// Reduce part[b * ncols + c] over b < nblocks for every column c, one warp
// per column, lane-strided then a fixed shuffle tree. Results to out[c].
__device__ __forceinline__ void reduce_partials(const double* part, int nblocks, int ncols, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wid; c < ncols; c += nw) {
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += __ldcg(&part[(int64_t)b * ncols + c]);
    s = warp_sum(s);
    if (lane == 0) out[c] = s;
  }
}

}  // namespace rk
