// Inexact deflation (csrc/dfl.cu): the block geometry, the subspace state and the coarse-vector
// kernels that the multigrid levels above it (csrc/mg.cu) share.
#pragma once

#include <algorithm>
#include <vector>

#include "sap.cuh"

namespace qxd {

constexpr int DFL_MAXVB = 256;  // sites per deflation block (threads of the block kernels)
constexpr int DFL_SLOTS = 9;    // self, then +mu, -mu for mu = 0..3

struct DflGeom {
  int b[4], n[4], stride[4];
  int vb, nb;
};

struct DflState {
  DflGeom dg;
  int ns = 0;
  double2* basis = nullptr;  // [ns][2][12][sv] FP64, the internal spinor layout, zero off its blocks
  float4* basis32 = nullptr; // [ns][2][6][sv] FP32 copy for applying P and P^+ to FP32 fields
  double2* A = nullptr;      // [nb][9][ns][ns]
  int* nbr = nullptr;        // [nb][9] block index per slot (device)
  std::vector<int> hnbr;     // host copy
  // coarse GCR work: vectors of n = nb ns complex (double2)
  double2* cw = nullptr;     // [2 m + 4][n]
  double* cpart = nullptr;   // reduction partials
  double* hcs = nullptr;     // pinned host scalars
  int m = 16;                // coarse GCR restart length
  double coarse_tol = 1e-2;  // relative residual of the coarse solve
  int coarse_maxiter = 64;
  i64 coarse_iters = 0;      // coarse iterations since set-up (statistics)
  i64 coarse_calls = 0;
  i64 epoch = -1;            // the lattice's field epoch at set-up (a later field change makes it stale)
  i64 gen = 0;               // set-up number (process-wide): a multigrid level built on it records it
};

// block coordinates of block index t (lexicographic, direction 3 fastest)
__host__ __device__ __forceinline__ void block_coords(const DflGeom& dg, int t, int kb[4]) {
  for (int mu = 3; mu >= 0; --mu) {
    kb[mu] = t % dg.n[mu];
    t /= dg.n[mu];
  }
}
__host__ __device__ __forceinline__ int block_index(const DflGeom& dg, const int kb[4]) {
  return ((kb[0] * dg.n[1] + kb[1]) * dg.n[2] + kb[2]) * dg.n[3] + kb[3];
}
__host__ __device__ __forceinline__ int block_colour(const int kb[4]) {
  return (kb[0] & 1) | ((kb[1] & 1) << 1) | ((kb[2] & 1) << 2) | ((kb[3] & 1) << 3);
}

// FP64 sums of NV values over the CTA (any blockDim <= 256); every thread receives the totals
template <int NV>
__device__ __forceinline__ void cta_sum(double v[NV], double* sh /* [NV][8 warps] */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double a = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    v[i] = a;
  }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[i * 8 + w] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double a = 0.0;
    for (int k = 0; k < nw; ++k) a += sh[i * 8 + k];  // fixed order: identical in every thread
    v[i] = a;
  }
}

inline int dfl_threads(const DflGeom& dg) { return (dg.vb + 31) / 32 * 32; }
inline int egrid(i64 n) { return (int)std::min<i64>((n + 255) / 256, 152 * 16); }


bool dfl_ready(const qxd_lattice* lat);

// kernels of csrc/dfl.cu used by csrc/mg.cu (V: the FP32 basis copy)
__global__ void __launch_bounds__(DFL_MAXVB) k_dfl_restrict(Geom g, DflGeom dg, int ns, const float4* __restrict__ V,
                                                            const float4* __restrict__ r, double2* __restrict__ f);
__global__ void __launch_bounds__(DFL_MAXVB) k_dfl_prolong(Geom g, DflGeom dg, int ns, const float4* __restrict__ V,
                                                           const double2* __restrict__ c, float4* __restrict__ z);

}  // namespace qxd
