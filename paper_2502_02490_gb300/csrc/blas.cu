// Fused BLAS-1 and FP64 global reductions.
//
// Reductions are deterministic: each block reduces a fixed grid-stride slice with warp shuffles,
// writes one partial per block into the lattice's partial buffer, and the last block to finish
// (ticket counter) sums the partials in block order and writes the result to a device scalar
// slot.  Accumulation is FP64 whatever the vector precision (the method keeps global inner
// products and norms in FP64).  Solver scalars (alpha, beta) are read from device slots, so a
// solver iteration needs no host round trip.
#include "qxd_internal.cuh"

namespace qxd {

static const int RB_THREADS = 256;

static int red_grid(qxd_lattice* lat, i64 n) {
  i64 b = (n + RB_THREADS - 1) / RB_THREADS;
  if (b > lat->red_blocks) b = lat->red_blocks;
  return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce NV values; thread 0 of the block returns them in v.
template <int NV>
__device__ __forceinline__ void block_sum(double v[NV]) {
  __shared__ double sh[NV][RB_THREADS / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    v[j] = warp_sum(v[j]);
    if (lane == 0) sh[j][w] = v[j];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double x = lane < (int)(blockDim.x >> 5) ? sh[j][lane] : 0.0;
      v[j] = warp_sum(x);
    }
  }
  __syncthreads();
}

// Store the block partials and let the last block finish the sum into scal[slot + j].
// Also runs `last_hook` in the last block after the sums are written.
template <int NV>
__device__ __forceinline__ bool finish_reduce(double v[NV], double* red, unsigned int* ticket, double* scal,
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
  if (!is_last) return false;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    s[j] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s[j] += __ldcg(red + (i64)j * gridDim.x + b);
  }
  block_sum<NV>(s);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) scal[slot + j] = s[j];
    *ticket = 0u;
  }
  return true;
}

__global__ void __launch_bounds__(RB_THREADS) k_norm2_64(const double2* __restrict__ a, i64 n, double* red,
                                                         unsigned int* ticket, double* scal, int slot) {
  double v[1] = {0.0};
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double2 x = a[i];
    v[0] += x.x * x.x + x.y * x.y;
  }
  block_sum<1>(v);
  finish_reduce<1>(v, red, ticket, scal, slot);
}

__global__ void __launch_bounds__(RB_THREADS) k_norm2_32(const float4* __restrict__ a, i64 n4, double* red,
                                                         unsigned int* ticket, double* scal, int slot) {
  double v[1] = {0.0};
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n4; i += (i64)gridDim.x * blockDim.x) {
    float4 x = a[i];
    v[0] += (double)x.x * x.x + (double)x.y * x.y + (double)x.z * x.z + (double)x.w * x.w;
  }
  block_sum<1>(v);
  finish_reduce<1>(v, red, ticket, scal, slot);
}

__global__ void __launch_bounds__(RB_THREADS) k_dot_64(const double2* __restrict__ a, const double2* __restrict__ b,
                                                       i64 n, double* red, unsigned int* ticket, double* scal,
                                                       int slot) {
  double v[2] = {0.0, 0.0};
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double2 x = a[i], y = b[i];
    v[0] += x.x * y.x + x.y * y.y;  // conj(x) y
    v[1] += x.x * y.y - x.y * y.x;
  }
  block_sum<2>(v);
  finish_reduce<2>(v, red, ticket, scal, slot);
}

__global__ void k_axpy_64(double re, double im, const double2* __restrict__ x, double2* __restrict__ y, i64 n) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double2 a = x[i], b = y[i];
    b.x += re * a.x - im * a.y;
    b.y += re * a.y + im * a.x;
    y[i] = b;
  }
}

__global__ void k_xpay_64(const double2* __restrict__ x, double a, double2* __restrict__ y, i64 n) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double2 u = x[i], v = y[i];
    y[i] = make_double2(u.x + a * v.x, u.y + a * v.y);
  }
}

__global__ void k_axpy_32(float a, const float4* __restrict__ x, float4* __restrict__ y, i64 n4) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n4; i += (i64)gridDim.x * blockDim.x) {
    float4 u = x[i], v = y[i];
    y[i] = make_float4(v.x + a * u.x, v.y + a * u.y, v.z + a * u.z, v.w + a * u.w);
  }
}

// y (FP64, [12][sv] double2) += x (FP32, [6][sv] float4)
__global__ void k_acc_f32_f64(i64 sv, i64 n4, const float4* __restrict__ x, double2* __restrict__ y) {
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n4; t += (i64)gridDim.x * blockDim.x) {
    i64 j = t / sv, cb = t - j * sv;
    float4 v = x[t];
    double2 a = y[(2 * j) * sv + cb], b = y[(2 * j + 1) * sv + cb];
    y[(2 * j) * sv + cb] = make_double2(a.x + v.x, a.y + v.y);
    y[(2 * j + 1) * sv + cb] = make_double2(b.x + v.z, b.y + v.w);
  }
}

// x += alpha p;  s -= alpha q;  scal[SC_SS] = ||s||^2, alpha = scal[SC_GAMMA] / scal[SC_QQ]
__global__ void __launch_bounds__(RB_THREADS) k_cg_xs_64(double2* __restrict__ x, const double2* __restrict__ p,
                                                         double2* __restrict__ s, const double2* __restrict__ q,
                                                         i64 n, double* red, unsigned int* ticket, double* scal) {
  double alpha = scal[SC_GAMMA] / scal[SC_QQ];
  double v[1] = {0.0};
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double2 xi = x[i], pi = p[i], si = s[i], qi = q[i];
    xi.x += alpha * pi.x;
    xi.y += alpha * pi.y;
    si.x -= alpha * qi.x;
    si.y -= alpha * qi.y;
    x[i] = xi;
    s[i] = si;
    v[0] += si.x * si.x + si.y * si.y;
  }
  block_sum<1>(v);
  finish_reduce<1>(v, red, ticket, scal, SC_SS);
}

__global__ void __launch_bounds__(RB_THREADS) k_cg_xs_32(float4* __restrict__ x, const float4* __restrict__ p,
                                                         float4* __restrict__ s, const float4* __restrict__ q,
                                                         i64 n4, double* red, unsigned int* ticket, double* scal) {
  float alpha = (float)(scal[SC_GAMMA] / scal[SC_QQ]);
  double v[1] = {0.0};
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n4; i += (i64)gridDim.x * blockDim.x) {
    float4 xi = x[i], pi = p[i], si = s[i], qi = q[i];
    xi.x += alpha * pi.x;
    xi.y += alpha * pi.y;
    xi.z += alpha * pi.z;
    xi.w += alpha * pi.w;
    si.x -= alpha * qi.x;
    si.y -= alpha * qi.y;
    si.z -= alpha * qi.z;
    si.w -= alpha * qi.w;
    x[i] = xi;
    s[i] = si;
    v[0] += (double)si.x * si.x + (double)si.y * si.y + (double)si.z * si.z + (double)si.w * si.w;
  }
  block_sum<1>(v);
  finish_reduce<1>(v, red, ticket, scal, SC_SS);
}

// p = r + beta p, beta = scal[SC_GAMMA_NEW] / scal[SC_GAMMA]; the last block then moves
// GAMMA_NEW into GAMMA (after every block has read both).
__device__ __forceinline__ void move_gamma(unsigned int* ticket, double* scal) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
    if (is_last) {
      scal[SC_GAMMA] = scal[SC_GAMMA_NEW];
      *ticket = 0u;
    }
  }
}

__global__ void __launch_bounds__(RB_THREADS) k_cg_p_64(const double2* __restrict__ r, double2* __restrict__ p,
                                                        i64 n, unsigned int* ticket, double* scal) {
  double beta = scal[SC_GAMMA_NEW] / scal[SC_GAMMA];
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double2 ri = r[i], pi = p[i];
    p[i] = make_double2(ri.x + beta * pi.x, ri.y + beta * pi.y);
  }
  move_gamma(ticket, scal);
}

__global__ void __launch_bounds__(RB_THREADS) k_cg_p_32(const float4* __restrict__ r, float4* __restrict__ p,
                                                        i64 n4, unsigned int* ticket, double* scal) {
  float beta = (float)(scal[SC_GAMMA_NEW] / scal[SC_GAMMA]);
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n4; i += (i64)gridDim.x * blockDim.x) {
    float4 ri = r[i], pi = p[i];
    p[i] = make_float4(ri.x + beta * pi.x, ri.y + beta * pi.y, ri.z + beta * pi.z, ri.w + beta * pi.w);
  }
  move_gamma(ticket, scal);
}

__global__ void k_set_scalar(double* scal, int slot, double v) { scal[slot] = v; }

#define RED_ARGS lat->red, lat->ticket, lat->scal

qxd_status blas_norm2_64(qxd_lattice* lat, const double2* a, i64 n, int slot) {
  k_norm2_64<<<red_grid(lat, n), RB_THREADS, 0, lat->stream>>>(a, n, RED_ARGS, slot);
  QXD_CHECK_LAUNCH(lat, "k_norm2_64");
  return QXD_OK;
}
qxd_status blas_norm2_32(qxd_lattice* lat, const float4* a, i64 n4, int slot) {
  k_norm2_32<<<red_grid(lat, n4), RB_THREADS, 0, lat->stream>>>(a, n4, RED_ARGS, slot);
  QXD_CHECK_LAUNCH(lat, "k_norm2_32");
  return QXD_OK;
}
qxd_status blas_dot_64(qxd_lattice* lat, const double2* a, const double2* b, i64 n, int slot) {
  k_dot_64<<<red_grid(lat, n), RB_THREADS, 0, lat->stream>>>(a, b, n, RED_ARGS, slot);
  QXD_CHECK_LAUNCH(lat, "k_dot_64");
  return QXD_OK;
}
qxd_status blas_axpy_64(qxd_lattice* lat, double re, double im, const double2* x, double2* y, i64 n) {
  k_axpy_64<<<red_grid(lat, n), RB_THREADS, 0, lat->stream>>>(re, im, x, y, n);
  QXD_CHECK_LAUNCH(lat, "k_axpy_64");
  return QXD_OK;
}
qxd_status blas_xpay_64(qxd_lattice* lat, const double2* x, double a, double2* y, i64 n) {
  k_xpay_64<<<red_grid(lat, n), RB_THREADS, 0, lat->stream>>>(x, a, y, n);
  QXD_CHECK_LAUNCH(lat, "k_xpay_64");
  return QXD_OK;
}
qxd_status blas_axpy_32(qxd_lattice* lat, float a, const float4* x, float4* y, i64 n4) {
  k_axpy_32<<<red_grid(lat, n4), RB_THREADS, 0, lat->stream>>>(a, x, y, n4);
  QXD_CHECK_LAUNCH(lat, "k_axpy_32");
  return QXD_OK;
}
qxd_status blas_acc_f32_into_f64(qxd_lattice* lat, const float4* x, double2* y, i64 n4) {
  k_acc_f32_f64<<<red_grid(lat, n4), RB_THREADS, 0, lat->stream>>>(lat->sv, n4, x, y);
  QXD_CHECK_LAUNCH(lat, "k_acc_f32_f64");
  return QXD_OK;
}
qxd_status cg_update_xs_64(qxd_lattice* lat, double2* x, const double2* p, double2* s, const double2* q, i64 n) {
  k_cg_xs_64<<<red_grid(lat, n), RB_THREADS, 0, lat->stream>>>(x, p, s, q, n, RED_ARGS);
  QXD_CHECK_LAUNCH(lat, "k_cg_xs_64");
  return QXD_OK;
}
qxd_status cg_update_xs_32(qxd_lattice* lat, float4* x, const float4* p, float4* s, const float4* q, i64 n4) {
  k_cg_xs_32<<<red_grid(lat, n4), RB_THREADS, 0, lat->stream>>>(x, p, s, q, n4, RED_ARGS);
  QXD_CHECK_LAUNCH(lat, "k_cg_xs_32");
  return QXD_OK;
}
qxd_status cg_update_p_64(qxd_lattice* lat, const double2* r, double2* p, i64 n) {
  k_cg_p_64<<<red_grid(lat, n), RB_THREADS, 0, lat->stream>>>(r, p, n, lat->ticket, lat->scal);
  QXD_CHECK_LAUNCH(lat, "k_cg_p_64");
  return QXD_OK;
}
qxd_status cg_update_p_32(qxd_lattice* lat, const float4* r, float4* p, i64 n4) {
  k_cg_p_32<<<red_grid(lat, n4), RB_THREADS, 0, lat->stream>>>(r, p, n4, lat->ticket, lat->scal);
  QXD_CHECK_LAUNCH(lat, "k_cg_p_32");
  return QXD_OK;
}
qxd_status set_scalar(qxd_lattice* lat, int slot, double v) {
  k_set_scalar<<<1, 1, 0, lat->stream>>>(lat->scal, slot, v);
  QXD_CHECK_LAUNCH(lat, "k_set_scalar");
  return QXD_OK;
}
qxd_status read_scalars(qxd_lattice* lat, int first, int count, double* out) {
  QXD_CUDA(lat, cudaMemcpyAsync(lat->hscal, lat->scal + first, sizeof(double) * count, cudaMemcpyDeviceToHost,
                                lat->stream));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  for (int i = 0; i < count; ++i) out[i] = lat->hscal[i];
  return QXD_OK;
}
qxd_status blas_copy(qxd_lattice* lat, void* dst, const void* src, size_t bytes) {
  QXD_CUDA(lat, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, lat->stream));
  return QXD_OK;
}
qxd_status blas_zero(qxd_lattice* lat, void* dst, size_t bytes) {
  QXD_CUDA(lat, cudaMemsetAsync(dst, 0, bytes, lat->stream));
  return QXD_OK;
}

}  // namespace qxd
