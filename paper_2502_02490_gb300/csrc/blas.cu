// Fused BLAS-1 and FP64 global reductions.
//
// Reductions are deterministic (reduce.cuh): fixed grid, per-block partials, the last block
// sums them in block order into a device scalar slot.  Accumulation is FP64 whatever the
// vector precision (global inner products and norms stay FP64).  Solver scalars (alpha, beta)
// are read from device slots, so a solver iteration needs no host round trip.  Each thread
// keeps UNROLL independent loads in flight.  For FP32 vectors the squares of one site (or of
// one unrolled group of 16 values) are summed in FP32 and all further accumulation is FP64; in
// the CG updates the sums within a thread and a warp are FP32 too, and the update coefficient is
// formed once per block.  FP64 arithmetic on GB300 runs at 1/64 of the FP32 rate, so FP64 work per
// element would make these bandwidth-bound kernels ALU-bound.  The CG updates work site by site so that they can
// also write the 16-bit copy (with its per-site scale) that the next 16-bit hop reads.
#include "reduce.cuh"

namespace qxd {

static const int RB = 256;   // threads per block
static const int UNROLL = 4;

static int red_grid(qxd_lattice* lat, i64 n) {
  i64 b = (n + (i64)RB * UNROLL - 1) / ((i64)RB * UNROLL);
  if (b > lat->red_blocks) b = lat->red_blocks;
  return (int)(b < 1 ? 1 : b);
}

static int site_grid(qxd_lattice* lat, i64 nsites) {
  i64 b = (nsites + RB - 1) / RB;
  if (b > lat->red_blocks) b = lat->red_blocks;
  return (int)(b < 1 ? 1 : b);
}

__global__ void __launch_bounds__(RB) k_norm2_64(const double2* __restrict__ a, i64 n, double* red,
                                                 unsigned int* ticket, double* scal, int slot) {
  double v[1] = {0.0};
  const i64 stride = (i64)gridDim.x * RB * UNROLL;
  for (i64 i0 = (i64)blockIdx.x * RB * UNROLL + threadIdx.x; i0 < n; i0 += stride) {
    double2 x[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) x[u] = (i0 + u * RB < n) ? a[i0 + u * RB] : make_double2(0.0, 0.0);
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) v[0] += x[u].x * x[u].x + x[u].y * x[u].y;
  }
  block_sum<1, RB>(v);
  finish_reduce<1, RB>(v, red, ticket, scal, slot);
}

__global__ void __launch_bounds__(RB) k_norm2_32(const float4* __restrict__ a, i64 n4, double* red,
                                                 unsigned int* ticket, double* scal, int slot) {
  double v[1] = {0.0};
  const i64 stride = (i64)gridDim.x * RB * UNROLL;
  for (i64 i0 = (i64)blockIdx.x * RB * UNROLL + threadIdx.x; i0 < n4; i0 += stride) {
    float4 x[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) x[u] = (i0 + u * RB < n4) ? a[i0 + u * RB] : make_float4(0.f, 0.f, 0.f, 0.f);
    // the 16 squares of one unrolled group are summed in FP32, everything beyond in FP64
    float g = 0.f;
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) g += (x[u].x * x[u].x + x[u].y * x[u].y) + (x[u].z * x[u].z + x[u].w * x[u].w);
    v[0] += (double)g;
  }
  block_sum<1, RB>(v);
  finish_reduce<1, RB>(v, red, ticket, scal, slot);
}

__global__ void __launch_bounds__(RB) k_dot_64(const double2* __restrict__ a, const double2* __restrict__ b, i64 n,
                                               double* red, unsigned int* ticket, double* scal, int slot) {
  double v[2] = {0.0, 0.0};
  const i64 stride = (i64)gridDim.x * RB * UNROLL;
  for (i64 i0 = (i64)blockIdx.x * RB * UNROLL + threadIdx.x; i0 < n; i0 += stride) {
    double2 x[UNROLL], y[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      bool ok = i0 + u * RB < n;
      x[u] = ok ? a[i0 + u * RB] : make_double2(0.0, 0.0);
      y[u] = ok ? b[i0 + u * RB] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      v[0] += x[u].x * y[u].x + x[u].y * y[u].y;  // conj(x) y
      v[1] += x[u].x * y[u].y - x[u].y * y[u].x;
    }
  }
  block_sum<2, RB>(v);
  finish_reduce<2, RB>(v, red, ticket, scal, slot);
}

__global__ void k_axpy_64(double re, double im, const double2* __restrict__ x, double2* __restrict__ y, i64 n) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double2 a = x[i], b = y[i];
    b.x += re * a.x - im * a.y;
    b.y += re * a.y + im * a.x;
    y[i] = b;
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

// 16-bit copy of one site's six float4 components with its per-site scale.
template <class FMT>
__device__ __forceinline__ void store_n16(const float4 v[6], uint2* __restrict__ o, float* __restrict__ on, i64 sv,
                                          i64 cb) {
  float m = 0.f;
#pragma unroll
  for (int j = 0; j < 6; ++j) m = fmaxf(m, fmaxf(fmaxf(fabsf(v[j].x), fabsf(v[j].y)), fmaxf(fabsf(v[j].z), fabsf(v[j].w))));
  const float inv = m > 0.f ? 1.f / m : 0.f;
  on[cb] = m;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    uint2 h;
    h.x = FMT::pack(v[j].x * inv, v[j].y * inv);
    h.y = FMT::pack(v[j].z * inv, v[j].w * inv);
    o[j * sv + cb] = h;
  }
}

__global__ void __launch_bounds__(RB) k_cg_xs_64(double2* __restrict__ x, const double2* __restrict__ p,
                                                 double2* __restrict__ s, const double2* __restrict__ q, i64 n,
                                                 double* red, unsigned int* ticket, double* scal) {
  const double alpha = scal[SC_GAMMA] / scal[SC_QQ];
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
  block_sum<1, RB>(v);
  finish_reduce<1, RB>(v, red, ticket, scal, SC_SS);
}

// scal[num] / scal[den] in FP64, formed once per block by thread 0 and shared as FP32 (an FP64
// division per thread would make a bandwidth-bound update ALU-bound on GB300)
__device__ __forceinline__ float block_ratio(const double* scal, int num, int den) {
  __shared__ float q;
  if (threadIdx.x == 0) q = (float)(scal[num] / scal[den]);
  __syncthreads();
  return q;
}

// x += alpha p; s -= alpha q; scal[SC_SS] = ||s||^2; optionally s16 = 16-bit copy of s.
// alpha = scal[SC_GAMMA] / scal[SC_QQ].  One thread per site (sv sites incl. zero padding).
template <class FMT, bool WR16>
__global__ void __launch_bounds__(RB) k_cg_xs_32(float4* __restrict__ x, const float4* __restrict__ p,
                                                 float4* __restrict__ s, const float4* __restrict__ q, i64 sv,
                                                 uint2* __restrict__ s16, float* __restrict__ s16n, double* red,
                                                 unsigned int* ticket, double* scal) {
  const float alpha = block_ratio(scal, SC_GAMMA, SC_QQ);
  float f[1] = {0.f};  // FP32 within the thread and the warp, FP64 beyond (block_sum_f32)
  for (i64 cb = blockIdx.x * (i64)blockDim.x + threadIdx.x; cb < sv; cb += (i64)gridDim.x * blockDim.x) {
    float4 sn[6];
    float g = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const i64 i = j * sv + cb;
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
      sn[j] = si;
      g += (si.x * si.x + si.y * si.y) + (si.z * si.z + si.w * si.w);
    }
    f[0] += g;
    if (WR16) store_n16<FMT>(sn, s16, s16n, sv, cb);
  }
  double v[1] = {0.0};
  block_sum_f32<1, RB>(f, v);
  finish_reduce<1, RB>(v, red, ticket, scal, SC_SS);
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

__global__ void __launch_bounds__(RB) k_cg_p_64(const double2* __restrict__ r, double2* __restrict__ p, i64 n,
                                                unsigned int* ticket, double* scal) {
  const double beta = scal[SC_GAMMA_NEW] / scal[SC_GAMMA];
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double2 ri = r[i], pi = p[i];
    p[i] = make_double2(ri.x + beta * pi.x, ri.y + beta * pi.y);
  }
  move_gamma(ticket, scal);
}

template <class FMT, bool WR16>
__global__ void __launch_bounds__(RB) k_cg_p_32(const float4* __restrict__ r, float4* __restrict__ p, i64 sv,
                                                uint2* __restrict__ p16, float* __restrict__ p16n,
                                                unsigned int* ticket, double* scal) {
  const float beta = block_ratio(scal, SC_GAMMA_NEW, SC_GAMMA);
  for (i64 cb = blockIdx.x * (i64)blockDim.x + threadIdx.x; cb < sv; cb += (i64)gridDim.x * blockDim.x) {
    float4 pn[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const i64 i = j * sv + cb;
      float4 ri = r[i], pi = p[i];
      pi = make_float4(ri.x + beta * pi.x, ri.y + beta * pi.y, ri.z + beta * pi.z, ri.w + beta * pi.w);
      p[i] = pi;
      pn[j] = pi;
    }
    if (WR16) store_n16<FMT>(pn, p16, p16n, sv, cb);
  }
  move_gamma(ticket, scal);
}

__global__ void k_set_scalar(double* scal, int slot, double v) { scal[slot] = v; }

#define RED_ARGS lat->red, lat->ticket, lat->scal

qxd_status blas_norm2_64(qxd_lattice* lat, const double2* a, i64 n, int slot) {
  k_norm2_64<<<red_grid(lat, n), RB, 0, lat->stream>>>(a, n, RED_ARGS, slot);
  QXD_CHECK_LAUNCH(lat, "k_norm2_64");
  return QXD_OK;
}
qxd_status blas_norm2_32(qxd_lattice* lat, const float4* a, i64 n4, int slot) {
  k_norm2_32<<<red_grid(lat, n4), RB, 0, lat->stream>>>(a, n4, RED_ARGS, slot);
  QXD_CHECK_LAUNCH(lat, "k_norm2_32");
  return QXD_OK;
}
qxd_status blas_dot_64(qxd_lattice* lat, const double2* a, const double2* b, i64 n, int slot) {
  k_dot_64<<<red_grid(lat, n), RB, 0, lat->stream>>>(a, b, n, RED_ARGS, slot);
  QXD_CHECK_LAUNCH(lat, "k_dot_64");
  return QXD_OK;
}
qxd_status blas_axpy_64(qxd_lattice* lat, double re, double im, const double2* x, double2* y, i64 n) {
  k_axpy_64<<<site_grid(lat, n), RB, 0, lat->stream>>>(re, im, x, y, n);
  QXD_CHECK_LAUNCH(lat, "k_axpy_64");
  return QXD_OK;
}
qxd_status blas_axpy_32(qxd_lattice* lat, float a, const float4* x, float4* y, i64 n4) {
  k_axpy_32<<<site_grid(lat, n4), RB, 0, lat->stream>>>(a, x, y, n4);
  QXD_CHECK_LAUNCH(lat, "k_axpy_32");
  return QXD_OK;
}
qxd_status blas_acc_f32_into_f64(qxd_lattice* lat, const float4* x, double2* y, i64 n4) {
  k_acc_f32_f64<<<site_grid(lat, n4), RB, 0, lat->stream>>>(lat->sv, n4, x, y);
  QXD_CHECK_LAUNCH(lat, "k_acc_f32_f64");
  return QXD_OK;
}
qxd_status cg_update_xs_64(qxd_lattice* lat, double2* x, const double2* p, double2* s, const double2* q, i64 n) {
  k_cg_xs_64<<<site_grid(lat, n), RB, 0, lat->stream>>>(x, p, s, q, n, RED_ARGS);
  QXD_CHECK_LAUNCH(lat, "k_cg_xs_64");
  return QXD_OK;
}
qxd_status cg_update_xs_32(qxd_lattice* lat, float4* x, const float4* p, float4* s, const float4* q, uint2* s16,
                           float* s16n, int bf16) {
  const i64 sv = lat->sv;
  const int g = site_grid(lat, sv);
  if (!s16)
    k_cg_xs_32<H16, false><<<g, RB, 0, lat->stream>>>(x, p, s, q, sv, nullptr, nullptr, RED_ARGS);
  else if (bf16)
    k_cg_xs_32<B16, true><<<g, RB, 0, lat->stream>>>(x, p, s, q, sv, s16, s16n, RED_ARGS);
  else
    k_cg_xs_32<H16, true><<<g, RB, 0, lat->stream>>>(x, p, s, q, sv, s16, s16n, RED_ARGS);
  QXD_CHECK_LAUNCH(lat, "k_cg_xs_32");
  return QXD_OK;
}
// The same updates on full fields [2][6][sv]: the kernels walk 6 planes of stride 2 sv, which
// visits every float4 of the field once (the update is elementwise, the norm a plain sum).
qxd_status cg_update_xs_32_full(qxd_lattice* lat, float4* x, const float4* p, float4* s, const float4* q) {
  const i64 st = 2 * lat->sv;
  k_cg_xs_32<H16, false><<<site_grid(lat, st), RB, 0, lat->stream>>>(x, p, s, q, st, nullptr, nullptr, RED_ARGS);
  QXD_CHECK_LAUNCH(lat, "k_cg_xs_32");
  return QXD_OK;
}
qxd_status cg_update_p_32_full(qxd_lattice* lat, const float4* r, float4* p) {
  const i64 st = 2 * lat->sv;
  k_cg_p_32<H16, false><<<site_grid(lat, st), RB, 0, lat->stream>>>(r, p, st, nullptr, nullptr, lat->ticket, lat->scal);
  QXD_CHECK_LAUNCH(lat, "k_cg_p_32");
  return QXD_OK;
}
qxd_status cg_update_p_64(qxd_lattice* lat, const double2* r, double2* p, i64 n) {
  k_cg_p_64<<<site_grid(lat, n), RB, 0, lat->stream>>>(r, p, n, lat->ticket, lat->scal);
  QXD_CHECK_LAUNCH(lat, "k_cg_p_64");
  return QXD_OK;
}
qxd_status cg_update_p_32(qxd_lattice* lat, const float4* r, float4* p, uint2* p16, float* p16n, int bf16) {
  const i64 sv = lat->sv;
  const int g = site_grid(lat, sv);
  if (!p16)
    k_cg_p_32<H16, false><<<g, RB, 0, lat->stream>>>(r, p, sv, nullptr, nullptr, lat->ticket, lat->scal);
  else if (bf16)
    k_cg_p_32<B16, true><<<g, RB, 0, lat->stream>>>(r, p, sv, p16, p16n, lat->ticket, lat->scal);
  else
    k_cg_p_32<H16, true><<<g, RB, 0, lat->stream>>>(r, p, sv, p16, p16n, lat->ticket, lat->scal);
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
