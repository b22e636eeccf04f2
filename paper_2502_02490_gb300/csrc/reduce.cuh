// Deterministic block and grid reductions shared by the BLAS-1 and hop kernels (FP64 beyond the
// warp; FP32 within a warp for the FP32-vector kernels).
//
// Each block reduces its values with warp shuffles and shared memory; thread 0 stores the
// block's partial in partial[j * gridDim.x + blockIdx.x]; the last block to finish (ticket
// counter) sums the partials in block order and writes scal[slot + j].  The summation order
// depends only on the grid, so results are reproducible run to run.
#pragma once

#include "qxd_internal.cuh"

namespace qxd {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce NV values (BLOCK threads); thread 0 holds the totals afterwards.
template <int NV, int BLOCK>
__device__ __forceinline__ void block_sum(double v[NV]) {
  __shared__ double sh[NV][BLOCK / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    v[j] = warp_sum(v[j]);
    if (lane == 0) sh[j][w] = v[j];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = warp_sum(lane < BLOCK / 32 ? sh[j][lane] : 0.0);
  }
  __syncthreads();
}

// Block-reduce NV FP32 values: sums over the 32 lanes of a warp in FP32, the warp partials and
// everything beyond in FP64 (FP64 runs at 1/64 of the FP32 rate on GB300, so an FP64 shuffle tree
// in every thread would dominate a bandwidth-bound kernel).  Thread 0 holds the totals afterwards.
template <int NV, int BLOCK>
__device__ __forceinline__ void block_sum_f32(const float f[NV], double v[NV]) {
  __shared__ double sh[NV][BLOCK / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    float x = f[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[j][w] = (double)x;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = warp_sum(lane < BLOCK / 32 ? sh[j][lane] : 0.0);
  }
  __syncthreads();
}

// Store the block partials; the last block sums them in order into scal[slot + j].
template <int NV, int BLOCK>
__device__ __forceinline__ void finish_reduce(double v[NV], double* red, unsigned int* ticket, double* scal,
                                              int slot) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) red[(i64)j * gridDim.x + blockIdx.x] = v[j];
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // the last block sums the partials in a fixed order, 8 independent loads in flight per thread
  constexpr int ILP = 8;
  double s[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const double* src = red + (i64)j * gridDim.x;
    double acc[ILP];
#pragma unroll
    for (int u = 0; u < ILP; ++u) acc[u] = 0.0;
    for (int b0 = threadIdx.x; b0 < (int)gridDim.x; b0 += BLOCK * ILP) {
#pragma unroll
      for (int u = 0; u < ILP; ++u) {
        const int b = b0 + u * BLOCK;
        acc[u] += b < (int)gridDim.x ? __ldcg(src + b) : 0.0;
      }
    }
    s[j] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  }
  block_sum<NV, BLOCK>(s);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) scal[slot + j] = s[j];
    *ticket = 0u;
  }
}

}  // namespace qxd
