// Fused vector kernels of BiCGStab on the even-odd system (FP32 vectors, FP64 reductions).
//
// BiCGStab for Dhat x = b (r_hat the fixed shadow residual):
//   v = Dhat p;  alpha = rho / <r_hat, v>;  s = r - alpha v;  t = Dhat s;
//   omega = <t, s> / <t, t>;  x += alpha p + omega s;  r = s - omega t;
//   rho' = <r_hat, r>;  beta = (rho' / rho)(alpha / omega);  p = r + beta (p - omega v).
// The complex scalars live in device slots (SC_RHO, SC_RV, SC_TS, SC_TT, SC_RR, SC_RN); each
// kernel recomputes alpha, omega, beta from them, so an iteration needs no host round trip.
// Kernels work site by site (one thread per site, six float4 per site) so they can also write
// the 16-bit copies (with per-site scale) that the next 16-bit Dhat reads; products are summed in
// FP32 within a thread and a warp and in FP64 beyond, and the coefficients are formed once per block.
//
// Multi-RHS: blockIdx.y selects the right-hand side.  Its vectors sit at base + rhs * rs
// (float4s), its scalars at scal + rhs * SC_N, its ticket at ticket + rhs and its partial sums
// at red + rhs * 3 * gridDim.x.  A right-hand side whose slot SC_ACTIVE is 0 is frozen (no
// vector update).  One right-hand side is gridDim.y = 1.
#include "reduce.cuh"

namespace qxd {

static const int BB = 256;

static dim3 bgrid(qxd_lattice* lat, int nrhs) {
  i64 b = (lat->sv + BB - 1) / BB;
  if (b > lat->red_blocks) b = lat->red_blocks;
  return dim3((unsigned)(b < 1 ? 1 : b), (unsigned)nrhs);
}

// Per-RHS views of the reduction state.
struct RhsView {
  double* red;
  unsigned int* ticket;
  double* scal;
  i64 off;  // float4 offset of this RHS's vectors
};

__device__ __forceinline__ RhsView rhs_view(double* red, unsigned int* ticket, double* scal, i64 rs) {
  const int r = blockIdx.y;
  RhsView v;
  v.red = red + (i64)r * 3 * gridDim.x;
  v.ticket = ticket + r;
  v.scal = scal + (i64)r * SC_N;
  v.off = (i64)r * rs;
  return v;
}

struct cd2 {
  double re, im;
};
__device__ __forceinline__ cd2 cdiv(cd2 a, cd2 b) {
  double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__device__ __forceinline__ cd2 cmul2(cd2 a, cd2 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// The BiCGStab coefficients of a block, formed once in FP64 by thread 0 from the device slots and
// shared as FP32 (FP64 runs at 1/64 of the FP32 rate on GB300: a complex division per thread
// would make these bandwidth-bound kernels ALU-bound).  KIND 0: -alpha; 1: alpha, omega;
// 2: beta, omega.  Returns false, uniformly over the block, for a frozen right-hand side.
template <int KIND>
__device__ __forceinline__ bool block_coefs(const double* scal, float c[4]) {
  __shared__ float sc[4];
  __shared__ int act;
  if (threadIdx.x == 0) {
    act = scal[SC_ACTIVE] != 0.0;
    const cd2 rho = {scal[SC_RHO], scal[SC_RHO + 1]};
    const cd2 alpha = cdiv(rho, {scal[SC_RV], scal[SC_RV + 1]});
    if (KIND == 0) {
      sc[0] = (float)-alpha.re;
      sc[1] = (float)-alpha.im;
    } else {
      const cd2 omega = {scal[SC_TS] / scal[SC_TT], scal[SC_TS + 1] / scal[SC_TT]};
      const cd2 a = KIND == 1 ? alpha : cmul2(cdiv({scal[SC_RR], scal[SC_RR + 1]}, rho), cdiv(alpha, omega));
      sc[0] = (float)a.re;
      sc[1] = (float)a.im;
      sc[2] = (float)omega.re;
      sc[3] = (float)omega.im;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) c[k] = sc[k];
  return act != 0;
}

__device__ __forceinline__ float4 caxpy4(float ar, float ai, float4 x, float4 y) {  // y + a x (two complex)
  return make_float4(y.x + ar * x.x - ai * x.y, y.y + ar * x.y + ai * x.x, y.z + ar * x.z - ai * x.w,
                     y.w + ar * x.w + ai * x.z);
}

template <class FMT>
__device__ __forceinline__ void store16(const float4 v[6], uint2* __restrict__ o, float* __restrict__ on, i64 sv,
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

// conj(a) b summed over the two complex numbers of a float4 pair
__device__ __forceinline__ void cdot4(float4 a, float4 b, float& re, float& im) {
  re += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
  im += a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
}

// Per-thread sums (over the thread's sites) and warp sums are FP32, block and grid sums FP64
// (block_sum_f32).

// scal[slot..slot+1] = <a, b>
__global__ void __launch_bounds__(BB) k_cdot_32(const float4* __restrict__ a, const float4* __restrict__ b, i64 sv,
                                                i64 rs, double* red0, unsigned int* ticket0, double* scal0, int slot) {
  const RhsView rv = rhs_view(red0, ticket0, scal0, rs);
  a += rv.off;
  b += rv.off;
  float f[2] = {0.f, 0.f};
  for (i64 cb = blockIdx.x * (i64)BB + threadIdx.x; cb < sv; cb += (i64)gridDim.x * BB) {
#pragma unroll
    for (int j = 0; j < 6; ++j) cdot4(a[j * sv + cb], b[j * sv + cb], f[0], f[1]);
  }
  double v[2] = {0.0, 0.0};
  block_sum_f32<2, BB>(f, v);
  finish_reduce<2, BB>(v, rv.red, rv.ticket, rv.scal, slot);
}

// s = r - alpha v, alpha = rho / <r_hat, v>; optional 16-bit s
template <class FMT, bool WR16>
__global__ void __launch_bounds__(BB) k_bicg_s(const float4* __restrict__ r, const float4* __restrict__ v,
                                               float4* __restrict__ s, uint2* __restrict__ s16, float* __restrict__ s16n,
                                               i64 sv, i64 rs, double* scal0) {
  float c[4];
  if (!block_coefs<0>(scal0 + (i64)blockIdx.y * SC_N, c)) return;
  r += (i64)blockIdx.y * rs;
  v += (i64)blockIdx.y * rs;
  s += (i64)blockIdx.y * rs;
  if (WR16) {  // 16-bit copies of a multi-RHS field: [rhs][6][sv] values, [rhs][sv] norms
    s16 += (i64)blockIdx.y * rs;
    s16n += (i64)blockIdx.y * sv;
  }
  const float ar = c[0], ai = c[1];
  for (i64 cb = blockIdx.x * (i64)BB + threadIdx.x; cb < sv; cb += (i64)gridDim.x * BB) {
    float4 o[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      o[j] = caxpy4(ar, ai, v[j * sv + cb], r[j * sv + cb]);
      s[j * sv + cb] = o[j];
    }
    if (WR16) store16<FMT>(o, s16, s16n, sv, cb);
  }
}

// scal[SC_TS..] = <t, s>, scal[SC_TT] = <t, t>
__global__ void __launch_bounds__(BB) k_bicg_ts(const float4* __restrict__ t, const float4* __restrict__ s, i64 sv,
                                                i64 rs, double* red0, unsigned int* ticket0, double* scal0) {
  const RhsView rv = rhs_view(red0, ticket0, scal0, rs);
  t += rv.off;
  s += rv.off;
  float f[3] = {0.f, 0.f, 0.f};
  for (i64 cb = blockIdx.x * (i64)BB + threadIdx.x; cb < sv; cb += (i64)gridDim.x * BB) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float4 a = t[j * sv + cb];
      cdot4(a, s[j * sv + cb], f[0], f[1]);
      f[2] += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
    }
  }
  double v[3] = {0.0, 0.0, 0.0};
  block_sum_f32<3, BB>(f, v);
  finish_reduce<3, BB>(v, rv.red, rv.ticket, rv.scal, SC_TS);  // SC_TS, SC_TS + 1, SC_TT = SC_TS + 2
}

// x += alpha p + omega s;  r = s - omega t;  scal[SC_RR..] = <r_hat, r>, scal[SC_RN] = ||r||^2
__global__ void __launch_bounds__(BB) k_bicg_xr(float4* __restrict__ x, const float4* __restrict__ p,
                                                const float4* __restrict__ s, const float4* __restrict__ t,
                                                const float4* __restrict__ rh, float4* __restrict__ r, i64 sv,
                                                i64 rs, double* red0, unsigned int* ticket0, double* scal0) {
  const RhsView rv = rhs_view(red0, ticket0, scal0, rs);
  float c[4];
  if (!block_coefs<1>(rv.scal, c)) return;  // uniform over the RHS's blocks: none of them takes part
  x += rv.off;
  p += rv.off;
  s += rv.off;
  t += rv.off;
  rh += rv.off;
  r += rv.off;
  const float a_r = c[0], a_i = c[1], w_r = c[2], w_i = c[3];
  float f[3] = {0.f, 0.f, 0.f};
  for (i64 cb = blockIdx.x * (i64)BB + threadIdx.x; cb < sv; cb += (i64)gridDim.x * BB) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const i64 i = j * sv + cb;
      float4 sj = s[i];
      x[i] = caxpy4(w_r, w_i, sj, caxpy4(a_r, a_i, p[i], x[i]));
      float4 rj = caxpy4(-w_r, -w_i, t[i], sj);
      r[i] = rj;
      cdot4(rh[i], rj, f[0], f[1]);
      f[2] += rj.x * rj.x + rj.y * rj.y + rj.z * rj.z + rj.w * rj.w;
    }
  }
  double v[3] = {0.0, 0.0, 0.0};
  block_sum_f32<3, BB>(f, v);
  finish_reduce<3, BB>(v, rv.red, rv.ticket, rv.scal, SC_RR);  // SC_RR, SC_RR + 1, SC_RN = SC_RR + 2
}

// p = r + beta (p - omega v), beta = (<r_hat,r> / rho)(alpha / omega); optional 16-bit p; the
// last block then sets rho = <r_hat, r> (after every block has read the old rho).
template <class FMT, bool WR16>
__global__ void __launch_bounds__(BB) k_bicg_p(const float4* __restrict__ r, const float4* __restrict__ v,
                                               float4* __restrict__ p, uint2* __restrict__ p16, float* __restrict__ p16n,
                                               i64 sv, i64 rs, unsigned int* ticket0, double* scal0) {
  double* scal = scal0 + (i64)blockIdx.y * SC_N;
  unsigned int* ticket = ticket0 + blockIdx.y;
  float c[4];
  if (!block_coefs<2>(scal, c)) return;
  r += (i64)blockIdx.y * rs;
  v += (i64)blockIdx.y * rs;
  p += (i64)blockIdx.y * rs;
  if (WR16) {  // as in k_bicg_s
    p16 += (i64)blockIdx.y * rs;
    p16n += (i64)blockIdx.y * sv;
  }
  const float b_r = c[0], b_i = c[1], w_r = c[2], w_i = c[3];
  for (i64 cb = blockIdx.x * (i64)BB + threadIdx.x; cb < sv; cb += (i64)gridDim.x * BB) {
    float4 o[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const i64 i = j * sv + cb;
      float4 q = caxpy4(-w_r, -w_i, v[i], p[i]);  // p - omega v
      o[j] = caxpy4(b_r, b_i, q, r[i]);
      p[i] = o[j];
    }
    if (WR16) store16<FMT>(o, p16, p16n, sv, cb);
  }
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    if (is_last) {
      scal[SC_RHO] = scal[SC_RR];
      scal[SC_RHO + 1] = scal[SC_RR + 1];
      *ticket = 0u;
    }
  }
}

// p = r (restart), optional 16-bit copy
template <class FMT, bool WR16>
__global__ void __launch_bounds__(BB) k_copy16(const float4* __restrict__ r, float4* __restrict__ p,
                                               uint2* __restrict__ p16, float* __restrict__ p16n, i64 sv) {
  r += (i64)blockIdx.y * 6 * sv;
  p += (i64)blockIdx.y * 6 * sv;
  for (i64 cb = blockIdx.x * (i64)BB + threadIdx.x; cb < sv; cb += (i64)gridDim.x * BB) {
    float4 o[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      o[j] = r[j * sv + cb];
      p[j * sv + cb] = o[j];
    }
    if (WR16) store16<FMT>(o, p16, p16n, sv, cb);
  }
}

// Reduction state of a launch over R.nrhs right-hand sides starting at R.r0.
struct RedState {
  double* red;
  unsigned int* ticket;
  double* scal;
};
static RedState red_state(qxd_lattice* lat, const Rhs& R) {
  if (!R.mr) return {lat->red, lat->ticket, lat->scal};
  const i64 gx = bgrid(lat, 1).x;
  return {lat->mr_red + (i64)R.r0 * 3 * gx, lat->mr_ticket + R.r0, lat->mr_scal + (i64)R.r0 * SC_N};
}

qxd_status bicg_cdot(qxd_lattice* lat, const float4* a, const float4* b, int slot, Rhs R) {
  RedState S = red_state(lat, R);
  k_cdot_32<<<bgrid(lat, R.nrhs), BB, 0, lat->stream>>>(a, b, lat->sv, R.rs, S.red, S.ticket, S.scal, slot);
  QXD_CHECK_LAUNCH(lat, "k_cdot_32");
  return QXD_OK;
}

qxd_status bicg_s(qxd_lattice* lat, const float4* r, const float4* v, float4* s, uint2* s16, float* s16n, int bf16,
                  Rhs R) {
  RedState S = red_state(lat, R);
  const dim3 g = bgrid(lat, R.nrhs);
  if (!s16)
    k_bicg_s<H16, false><<<g, BB, 0, lat->stream>>>(r, v, s, nullptr, nullptr, lat->sv, R.rs, S.scal);
  else if (bf16)
    k_bicg_s<B16, true><<<g, BB, 0, lat->stream>>>(r, v, s, s16, s16n, lat->sv, R.rs, S.scal);
  else
    k_bicg_s<H16, true><<<g, BB, 0, lat->stream>>>(r, v, s, s16, s16n, lat->sv, R.rs, S.scal);
  QXD_CHECK_LAUNCH(lat, "k_bicg_s");
  return QXD_OK;
}

qxd_status bicg_ts(qxd_lattice* lat, const float4* t, const float4* s, Rhs R) {
  RedState S = red_state(lat, R);
  k_bicg_ts<<<bgrid(lat, R.nrhs), BB, 0, lat->stream>>>(t, s, lat->sv, R.rs, S.red, S.ticket, S.scal);
  QXD_CHECK_LAUNCH(lat, "k_bicg_ts");
  return QXD_OK;
}

qxd_status bicg_xr(qxd_lattice* lat, float4* x, const float4* p, const float4* s, const float4* t, const float4* rh,
                   float4* r, Rhs R) {
  RedState S = red_state(lat, R);
  k_bicg_xr<<<bgrid(lat, R.nrhs), BB, 0, lat->stream>>>(x, p, s, t, rh, r, lat->sv, R.rs, S.red, S.ticket, S.scal);
  QXD_CHECK_LAUNCH(lat, "k_bicg_xr");
  return QXD_OK;
}

qxd_status bicg_p(qxd_lattice* lat, const float4* r, const float4* v, float4* p, uint2* p16, float* p16n, int bf16,
                  Rhs R) {
  RedState S = red_state(lat, R);
  const dim3 g = bgrid(lat, R.nrhs);
  if (!p16)
    k_bicg_p<H16, false><<<g, BB, 0, lat->stream>>>(r, v, p, nullptr, nullptr, lat->sv, R.rs, S.ticket, S.scal);
  else if (bf16)
    k_bicg_p<B16, true><<<g, BB, 0, lat->stream>>>(r, v, p, p16, p16n, lat->sv, R.rs, S.ticket, S.scal);
  else
    k_bicg_p<H16, true><<<g, BB, 0, lat->stream>>>(r, v, p, p16, p16n, lat->sv, R.rs, S.ticket, S.scal);
  QXD_CHECK_LAUNCH(lat, "k_bicg_p");
  return QXD_OK;
}

__global__ void k_set_at(double* p, double v) { *p = v; }

qxd_status set_scalar_at(qxd_lattice* lat, double* p, double v) {
  k_set_at<<<1, 1, 0, lat->stream>>>(p, v);
  QXD_CHECK_LAUNCH(lat, "k_set_at");
  return QXD_OK;
}

qxd_status ensure_mrhs(qxd_lattice* lat, int n) {
  if (lat->mr_cap >= n) return QXD_OK;
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  if (lat->mr_red) cudaFree(lat->mr_red);
  if (lat->mr_ticket) cudaFree(lat->mr_ticket);
  if (lat->mr_scal) cudaFree(lat->mr_scal);
  if (lat->mr_hscal) cudaFreeHost(lat->mr_hscal);
  lat->mr_red = nullptr;
  lat->mr_ticket = nullptr;
  lat->mr_scal = nullptr;
  lat->mr_hscal = nullptr;
  lat->mr_cap = 0;
  const i64 gx = bgrid(lat, 1).x;
  QXD_CUDA(lat, cudaMalloc((void**)&lat->mr_red, sizeof(double) * 3 * gx * n));
  QXD_CUDA(lat, cudaMalloc((void**)&lat->mr_ticket, sizeof(unsigned int) * n));
  QXD_CUDA(lat, cudaMalloc((void**)&lat->mr_scal, sizeof(double) * SC_N * n));
  QXD_CUDA(lat, cudaMallocHost((void**)&lat->mr_hscal, sizeof(double) * SC_N * n));
  QXD_CUDA(lat, cudaMemsetAsync(lat->mr_ticket, 0, sizeof(unsigned int) * n, lat->stream));
  QXD_CUDA(lat, cudaMemsetAsync(lat->mr_scal, 0, sizeof(double) * SC_N * n, lat->stream));
  lat->mr_cap = n;
  return QXD_OK;
}

qxd_status bicg_copy(qxd_lattice* lat, const float4* r, float4* p, uint2* p16, float* p16n, int bf16) {
  const dim3 g = bgrid(lat, 1);
  if (!p16)
    k_copy16<H16, false><<<g, BB, 0, lat->stream>>>(r, p, nullptr, nullptr, lat->sv);
  else if (bf16)
    k_copy16<B16, true><<<g, BB, 0, lat->stream>>>(r, p, p16, p16n, lat->sv);
  else
    k_copy16<H16, true><<<g, BB, 0, lat->stream>>>(r, p, p16, p16n, lat->sv);
  QXD_CHECK_LAUNCH(lat, "k_copy16");
  return QXD_OK;
}

}  // namespace qxd
