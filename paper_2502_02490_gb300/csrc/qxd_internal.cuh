// Internal types of libqxd: lattice geometry, device field layouts, precision accessors.
//
// Device layout (structure of arrays, one "plane" per component, stride sv >= Vh, padded to a
// multiple of 64 sites; padding entries stay zero):
//   FP64 spinor, one parity : double2 [12][sv]        component k = 3*alpha + a
//   FP32 spinor, one parity : float4  [6][sv]         components (2j, 2j+1)
//   16-bit spinor, one parity: uint2  [6][sv] + float norm [sv]   value = h * norm
//   links  : [parity][mu][9][sv]  (double2 / float2 / 32-bit half2-or-bf162), entry 3*row + col
//   clover : [parity][block][..][sv], 36 reals per block in the 36-real packing of Sec. 4.1.3
//            (double2 x18 / float4 x9 / uint2 x9 + float norm [parity][block][sv])
// A site of parity p with lexicographic index Lambda has checkerboard index cb = floor(Lambda/2),
// the openQxD in-parity index of Eq. ipt with one block.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qxd.h"

namespace qxd {

typedef int64_t i64;

// ------------------------------------------------------------------------------------------
// Geometry: pure index functions (no lookup tables), Sec. 4.1.1
// ------------------------------------------------------------------------------------------
// Division by a constant d >= 2 for 0 <= n < 2^31: with s = ceil(log2 d) and
// m = ceil(2^(31+s) / d) (< 2^32), n / d = umulhi(n, m) >> (s - 1).  The rounding error of m
// adds less than 2^-s <= 1/d to n/d, which cannot carry past the next integer.
struct FastDiv {
  uint32_t d, m, s1;
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t s = 0;
  while ((1ull << s) < d) ++s;
  unsigned long long m = ((1ull << (31 + s)) + d - 1) / d;
  FastDiv f;
  f.d = d;
  f.m = (uint32_t)m;
  f.s1 = s - 1;
  return f;
}

__host__ __device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
  return __umulhi(n, f.m) >> f.s1;
#else
  return (uint32_t)(((unsigned long long)n * f.m) >> 32) >> f.s1;
#endif
}

struct Geom {
  int L[4];    // extents on the device lattice (x doubled for C*)
  int shift;   // C*: physical L1 (mirror offset); 0 without C*
  int anti;    // 1: antiperiodic in time
  i64 Vh;      // sites per parity
  i64 sv;      // plane stride
  FastDiv dL1, dL2, dL3;  // divisions by L1, L2, L3 (V < 2^31)
  int B[4];    // cache-block extents of the IPT boundary order (B = L: one block)
};

// Eq. ipt with cache blocks: the boundary index of site x on a lattice of extents L with blocks
// B (each B_mu divides L_mu): floor((V_B Lambda(n, N_B) + Lambda(b, B)) / 2) + P(x) V / 2, with
// n = floor(x / B) the block and b = x mod B the site within it.  A pure function, no table.
__host__ __device__ __forceinline__ i64 ipt_index(const int L[4], const int B[4], const int x[4]) {
  i64 lam_n = 0, lam_b = 0, VB = 1, V = 1;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    lam_n = lam_n * (L[mu] / B[mu]) + x[mu] / B[mu];
    lam_b = lam_b * B[mu] + x[mu] % B[mu];
    VB *= B[mu];
    V *= L[mu];
  }
  const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
  return (VB * lam_n + lam_b) / 2 + (i64)par * (V / 2);
}

// Inverse of ipt_index: the site of boundary index i.  Of the two blocked lexicographic indices
// 2k and 2k + 1 (k = i - P V/2) exactly one has parity P.
__host__ __device__ __forceinline__ void ipt_coords(const int L[4], const int B[4], i64 i, int x[4]) {
  i64 VB = 1, V = 1;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    VB *= B[mu];
    V *= L[mu];
  }
  const int par = i >= V / 2 ? 1 : 0;
  const i64 k = i - (i64)par * (V / 2);
  for (int c = 0; c < 2; ++c) {
    const i64 lam = 2 * k + c;
    i64 ln = lam / VB, lb = lam % VB;
#pragma unroll
    for (int mu = 3; mu >= 0; --mu) {
      const int nb = L[mu] / B[mu];
      x[mu] = (int)(ln % nb) * B[mu] + (int)(lb % B[mu]);
      ln /= nb;
      lb /= B[mu];
    }
    if (((x[0] + x[1] + x[2] + x[3]) & 1) == par) return;
  }
}

__host__ __device__ __forceinline__ i64 lexi(const Geom& g, const int x[4]) {
  return (((i64)x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
}

// Coordinates of the site with checkerboard index cb and parity par.  Lambda = 2 cb or
// 2 cb + 1; the two candidates differ only in x3 (L3 is even), and the parity decides.
__host__ __device__ __forceinline__ void cb_coords(const Geom& g, i64 cb, int par, int x[4]) {
  i64 lam = 2 * cb;
  x[3] = (int)(lam % g.L[3]);
  i64 t = lam / g.L[3];
  x[2] = (int)(t % g.L[2]);
  t /= g.L[2];
  x[1] = (int)(t % g.L[1]);
  x[0] = (int)(t / g.L[1]);
  if (((x[0] + x[1] + x[2] + x[3]) & 1) != par) x[3] += 1;
}

// 32-bit version for V < 2^31 using the precomputed divisions.
__device__ __forceinline__ void cb_coords32(const Geom& g, uint32_t cb, int par, int x[4]) {
  uint32_t lam = 2u * cb;
  uint32_t q1 = fdiv(lam, g.dL3);
  x[3] = (int)(lam - q1 * g.dL3.d);
  uint32_t q2 = fdiv(q1, g.dL2);
  x[2] = (int)(q1 - q2 * g.dL2.d);
  uint32_t q3 = fdiv(q2, g.dL1);
  x[1] = (int)(q2 - q3 * g.dL1.d);
  x[0] = (int)q3;
  if (((x[0] + x[1] + x[2] + x[3]) & 1) != par) x[3] += 1;
}

// Checkerboard index of x + dir * mu_hat (32-bit); sets crossed on a wrap in direction mu.
__device__ __forceinline__ uint32_t nbr_cb32(const Geom& g, const int x[4], int mu, int dir, bool& crossed) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[mu] += dir;
  crossed = false;
  if (y[mu] >= g.L[mu]) {
    y[mu] = 0;
    crossed = true;
  } else if (y[mu] < 0) {
    y[mu] = g.L[mu] - 1;
    crossed = true;
  }
  if (crossed && g.shift && mu >= 2) {
    y[1] += g.shift;
    if (y[1] >= g.L[1]) y[1] -= g.L[1];
  }
  return ((((uint32_t)y[0] * g.L[1] + y[1]) * g.L[2] + y[2]) * g.L[3] + y[3]) >> 1;
}

// Checkerboard index of x + dir * mu_hat; `crossed` reports a wrap in direction mu.  With C*,
// a wrap in y or z lands on the mirror copy: x1 -> x1 + shift (mod 2 shift), Sec. 4.2.
__host__ __device__ __forceinline__ i64 nbr_cb(const Geom& g, const int x[4], int mu, int dir,
                                               bool& crossed) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[mu] += dir;
  crossed = false;
  if (y[mu] >= g.L[mu]) {
    y[mu] = 0;
    crossed = true;
  } else if (y[mu] < 0) {
    y[mu] = g.L[mu] - 1;
    crossed = true;
  }
  if (crossed && g.shift && mu >= 2) {
    y[1] += g.shift;
    if (y[1] >= g.L[1]) y[1] -= g.L[1];
  }
  return lexi(g, y) >> 1;
}

// ------------------------------------------------------------------------------------------
// Complex arithmetic
// ------------------------------------------------------------------------------------------
template <typename T>
struct cplx {
  T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ cplx<T> mk(T r, T i) {
  cplx<T> c;
  c.re = r;
  c.im = i;
  return c;
}
template <typename T>
__device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cplx<T> operator*(T s, cplx<T> a) { return mk(s * a.re, s * a.im); }
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// conj(a) * b
template <typename T>
__device__ __forceinline__ cplx<T> cjmul(cplx<T> a, cplx<T> b) {
  return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// s + a b and s + conj(a) b as four fused multiply-adds (accumulating into s directly: one
// rounding per product term, no separate products and additions)
template <typename T>
__device__ __forceinline__ cplx<T> cmac(cplx<T> s, cplx<T> a, cplx<T> b) {
  T re = fma(a.re, b.re, s.re), im = fma(a.re, b.im, s.im);
  re = fma(-a.im, b.im, re);
  im = fma(a.im, b.re, im);
  return mk(re, im);
}
template <typename T>
__device__ __forceinline__ cplx<T> cjmac(cplx<T> s, cplx<T> a, cplx<T> b) {
  T re = fma(a.re, b.re, s.re), im = fma(a.re, b.im, s.im);
  re = fma(a.im, b.im, re);
  im = fma(-a.im, b.re, im);
  return mk(re, im);
}
template <typename T>
__device__ __forceinline__ cplx<T> timesI(cplx<T> a) { return mk(-a.im, a.re); }
template <typename T>
__device__ __forceinline__ cplx<T> neg(cplx<T> a) { return mk(-a.re, -a.im); }

// ------------------------------------------------------------------------------------------
// 16-bit storage helpers
// ------------------------------------------------------------------------------------------
struct H16 {  // IEEE half
  static __device__ __forceinline__ float lo(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
  static __device__ __forceinline__ float hi(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    return (uint32_t)__half_as_ushort(__float2half_rn(a)) | ((uint32_t)__half_as_ushort(__float2half_rn(b)) << 16);
  }
};
struct B16 {  // bfloat16
  static __device__ __forceinline__ float lo(uint32_t w) { return __uint_as_float(w << 16); }
  static __device__ __forceinline__ float hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
  }
};

// ------------------------------------------------------------------------------------------
// Spinor accessors (one parity)
// ------------------------------------------------------------------------------------------
struct SpinorF64 {
  typedef double real;
  struct Raw {
    double2 v[12];
  };
  double2* p;
  i64 sv;
  __device__ __forceinline__ Raw fetch(uint32_t cb) const {
    Raw r;
#pragma unroll
    for (int k = 0; k < 12; ++k) r.v[k] = __ldg(p + k * sv + cb);
    return r;
  }
  // unscaled components; returns the scale (1 here)
  __device__ __forceinline__ double decode(const Raw& r, cplx<double> s[12]) const {
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = mk(r.v[k].x, r.v[k].y);
    return 1.0;
  }
  __device__ __forceinline__ void load(i64 cb, cplx<double> s[12]) const {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 v = __ldg(p + k * sv + cb);
      s[k] = mk(v.x, v.y);
    }
  }
  template <typename T>
  __device__ __forceinline__ void store(i64 cb, const cplx<T> s[12]) const {
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k * sv + cb] = make_double2((double)s[k].re, (double)s[k].im);
  }
};

struct SpinorF32 {
  typedef float real;
  struct Raw {
    float4 v[6];
  };
  float4* p;
  i64 sv;
  __device__ __forceinline__ Raw fetch(uint32_t cb) const {
    Raw r;
#pragma unroll
    for (int j = 0; j < 6; ++j) r.v[j] = __ldg(p + j * sv + cb);
    return r;
  }
  __device__ __forceinline__ float decode(const Raw& r, cplx<float> s[12]) const {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      s[2 * j] = mk(r.v[j].x, r.v[j].y);
      s[2 * j + 1] = mk(r.v[j].z, r.v[j].w);
    }
    return 1.0f;
  }
  __device__ __forceinline__ void load(i64 cb, cplx<float> s[12]) const {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float4 v = __ldg(p + j * sv + cb);
      s[2 * j] = mk(v.x, v.y);
      s[2 * j + 1] = mk(v.z, v.w);
    }
  }
  template <typename T>
  __device__ __forceinline__ void store(i64 cb, const cplx<T> s[12]) const {
#pragma unroll
    for (int j = 0; j < 6; ++j)
      p[j * sv + cb] = make_float4((float)s[2 * j].re, (float)s[2 * j].im, (float)s[2 * j + 1].re,
                                   (float)s[2 * j + 1].im);
  }
};

// 16-bit spinor with one FP32 scale per site: value = stored * norm, norm = max |component|.
template <class FMT>
struct SpinorN16 {
  typedef float real;
  struct Raw {
    uint2 v[6];
    float n;
  };
  uint2* p;
  float* nrm;
  i64 sv;
  __device__ __forceinline__ Raw fetch(uint32_t cb) const {
    Raw r;
#pragma unroll
    for (int j = 0; j < 6; ++j) r.v[j] = __ldg(p + j * sv + cb);
    r.n = __ldg(nrm + cb);
    return r;
  }
  // stored (unscaled) components; the caller applies the returned per-site scale
  __device__ __forceinline__ float decode(const Raw& r, cplx<float> s[12]) const {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      s[2 * j] = mk(FMT::lo(r.v[j].x), FMT::hi(r.v[j].x));
      s[2 * j + 1] = mk(FMT::lo(r.v[j].y), FMT::hi(r.v[j].y));
    }
    return r.n;
  }
  __device__ __forceinline__ void load(i64 cb, cplx<float> s[12]) const {
    float n = __ldg(nrm + cb);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      uint2 v = __ldg(p + j * sv + cb);
      s[2 * j] = mk(n * FMT::lo(v.x), n * FMT::hi(v.x));
      s[2 * j + 1] = mk(n * FMT::lo(v.y), n * FMT::hi(v.y));
    }
  }
  template <typename T>
  __device__ __forceinline__ void store(i64 cb, const cplx<T> s[12]) const {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf((float)s[k].re), fabsf((float)s[k].im)));
    float inv = m > 0.f ? 1.0f / m : 0.f;
    nrm[cb] = m;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      uint2 v;
      v.x = FMT::pack((float)s[2 * j].re * inv, (float)s[2 * j].im * inv);
      v.y = FMT::pack((float)s[2 * j + 1].re * inv, (float)s[2 * j + 1].im * inv);
      p[j * sv + cb] = v;
    }
  }
};

// ------------------------------------------------------------------------------------------
// Link accessors: [parity][mu][9][sv]
// ------------------------------------------------------------------------------------------
struct LinkF64 {
  typedef double real;
  struct Raw {
    double2 w[9];
  };
  const double2* p;
  i64 sv;
  __device__ __forceinline__ Raw fetch(int par, int mu, uint32_t cb) const {
    const double2* b = p + (i64)((par * 4 + mu) * 9) * sv + cb;
    Raw r;
#pragma unroll
    for (int k = 0; k < 9; ++k) r.w[k] = __ldg(b + k * sv);
    return r;
  }
  __device__ __forceinline__ void decode(const Raw& r, cplx<double> u[9]) const {
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = mk(r.w[k].x, r.w[k].y);
  }
  __device__ __forceinline__ void load(int par, int mu, i64 cb, cplx<double> u[9]) const {
    const double2* b = p + (i64)((par * 4 + mu) * 9) * sv + cb;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 v = __ldg(b + k * sv);
      u[k] = mk(v.x, v.y);
    }
  }
};
struct LinkF32 {
  typedef float real;
  struct Raw {
    float2 w[9];
  };
  const float2* p;
  i64 sv;
  __device__ __forceinline__ Raw fetch(int par, int mu, uint32_t cb) const {
    const float2* b = p + (i64)((par * 4 + mu) * 9) * sv + cb;
    Raw r;
#pragma unroll
    for (int k = 0; k < 9; ++k) r.w[k] = __ldg(b + k * sv);
    return r;
  }
  __device__ __forceinline__ void decode(const Raw& r, cplx<float> u[9]) const {
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = mk(r.w[k].x, r.w[k].y);
  }
  __device__ __forceinline__ void load(int par, int mu, i64 cb, cplx<float> u[9]) const {
    const float2* b = p + (i64)((par * 4 + mu) * 9) * sv + cb;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float2 v = __ldg(b + k * sv);
      u[k] = mk(v.x, v.y);
    }
  }
};
// 16-bit links (one 32-bit word, a complex pair, per entry): each (parity, direction) owns 9 sv
// words; a site's entries 0..3 form one 16-byte group at word 4 cb, entries 4..7 one at
// 4 sv + 4 cb, entry 8 sits at 8 sv + cb -- three loads per link instead of nine.
__host__ __device__ __forceinline__ i64 link16_index(i64 pm, i64 sv, int k, i64 cb) {  // pm = par * 4 + mu
  const i64 b = pm * 9 * sv;
  return k < 4 ? b + 4 * cb + k : k < 8 ? b + 4 * sv + 4 * cb + (k - 4) : b + 8 * sv + cb;
}

template <class FMT>
struct Link16 {
  typedef float real;
  struct Raw {
    uint32_t w[9];
  };
  const uint32_t* p;
  i64 sv;
  __device__ __forceinline__ Raw fetch(int par, int mu, uint32_t cb) const {
    const uint32_t* b = p + (i64)((par * 4 + mu) * 9) * sv;
    const uint4 a = __ldg((const uint4*)b + cb), c = __ldg((const uint4*)(b + 4 * sv) + cb);
    Raw r;
    r.w[0] = a.x;
    r.w[1] = a.y;
    r.w[2] = a.z;
    r.w[3] = a.w;
    r.w[4] = c.x;
    r.w[5] = c.y;
    r.w[6] = c.z;
    r.w[7] = c.w;
    r.w[8] = __ldg(b + 8 * sv + cb);
    return r;
  }
  __device__ __forceinline__ void decode(const Raw& r, cplx<float> u[9]) const {
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = mk(FMT::lo(r.w[k]), FMT::hi(r.w[k]));
  }
  __device__ __forceinline__ void words(const Raw& r, uint32_t w[9]) const {  // the stored 16-bit pairs
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = r.w[k];
  }
  __device__ __forceinline__ void load(int par, int mu, i64 cb, cplx<float> u[9]) const {
    const Raw r = fetch(par, mu, (uint32_t)cb);
    decode(r, u);
  }
};

// ------------------------------------------------------------------------------------------
// Clover accessors: 36 reals per (parity, block, site)
// ------------------------------------------------------------------------------------------
struct CloverF64 {
  typedef double real;
  struct Raw {};  // no epilogue prefetch for FP64
  const double2* p;
  i64 sv;
  __device__ __forceinline__ void load(int par, int blk, i64 cb, double r[36]) const {
    const double2* b = p + (i64)((par * 2 + blk) * 18) * sv + cb;
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      double2 v = __ldg(b + k * sv);
      r[2 * k] = v.x;
      r[2 * k + 1] = v.y;
    }
  }
};
struct CloverF32 {
  typedef float real;
  struct Raw {};  // no epilogue prefetch for FP32
  const float4* p;
  i64 sv;
  __device__ __forceinline__ void load(int par, int blk, i64 cb, float r[36]) const {
    const float4* b = p + (i64)((par * 2 + blk) * 9) * sv + cb;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float4 v = __ldg(b + k * sv);
      r[4 * k] = v.x;
      r[4 * k + 1] = v.y;
      r[4 * k + 2] = v.z;
      r[4 * k + 3] = v.w;
    }
  }
};
template <class FMT>
struct Clover16 {
  typedef float real;
  struct Raw {  // both chirality blocks of one site
    uint2 v[2][9];
    float n[2];
  };
  const uint2* p;
  const float* nrm;  // [parity][block][sv]
  i64 sv;
  __device__ __forceinline__ Raw fetch(int par, uint32_t cb) const {
    Raw r;
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
      const uint2* b = p + (i64)((par * 2 + blk) * 9) * sv + cb;
#pragma unroll
      for (int k = 0; k < 9; ++k) r.v[blk][k] = __ldg(b + k * sv);
      r.n[blk] = __ldg(nrm + (i64)(par * 2 + blk) * sv + cb);
    }
    return r;
  }
  __device__ __forceinline__ void decode(const Raw& r, int blk, float o[36]) const {
    const float n = r.n[blk];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      uint2 v = r.v[blk][k];
      o[4 * k] = n * FMT::lo(v.x);
      o[4 * k + 1] = n * FMT::hi(v.x);
      o[4 * k + 2] = n * FMT::lo(v.y);
      o[4 * k + 3] = n * FMT::hi(v.y);
    }
  }
  __device__ __forceinline__ void load(int par, int blk, i64 cb, float r[36]) const {
    const uint2* b = p + (i64)((par * 2 + blk) * 9) * sv + cb;
    float n = __ldg(nrm + (i64)(par * 2 + blk) * sv + cb);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      uint2 v = __ldg(b + k * sv);
      r[4 * k] = n * FMT::lo(v.x);
      r[4 * k + 1] = n * FMT::hi(v.x);
      r[4 * k + 2] = n * FMT::lo(v.y);
      r[4 * k + 3] = n * FMT::hi(v.y);
    }
  }
};

// y = M x for the Hermitian 6x6 block M packed in 36 reals (diagonal, then upper row-major).
template <typename R>
__device__ __forceinline__ void herm6_apply(const R r[36], const cplx<R> x[6], cplx<R> y[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] = r[i] * x[i];
  int k = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      cplx<R> c = mk(r[6 + 2 * k], r[7 + 2 * k]);
      y[i] = cmac(y[i], c, x[j]);
      y[j] = cjmac(y[j], c, x[i]);
      ++k;
    }
  }
}

// ------------------------------------------------------------------------------------------
// The lattice object (host side)
// ------------------------------------------------------------------------------------------
enum {
  KSTAT_F64 = 0,
  KSTAT_F32 = 1,
  KSTAT_F16N = 2,
  KSTAT_BF16N = 3,
  KSTAT_F32_MRHS = 4,
  KSTAT_BATCH = 5,
  KSTAT_PTC_TC = 6,   // tensor-core PTC layer
  KSTAT_PTC_F32 = 7,  // FP32 CUDA-core PTC layer
  KSTAT_N16_MRHS = 8, // 16-bit multi-RHS hop
  KSTAT_SAP = 9,      // SAP block minimal-residual sweep
  KSTAT_MR_BLAS = 10, // vector kernels of the multi-RHS BiCGStab
  KSTAT_N = 11
};

// Device scalar slots used by the solvers and reductions.
enum {
  SC_GAMMA = 0, SC_GAMMA_NEW, SC_QQ, SC_SS, SC_TMP0, SC_TMP1, SC_TMP2, SC_TMP3,
  // BiCGStab: complex pairs (re, im) at SC_RHO, SC_RV, SC_TS, SC_RR; reals SC_TT = SC_TS + 2,
  // SC_RN = SC_RR + 2 (written together by 3-value reductions)
  SC_RHO = 8, SC_RV = 10, SC_TS = 12, SC_TT = 14, SC_RR = 15, SC_RN = 17,
  SC_ACTIVE = 20,  // 1.0 while a right-hand side iterates, 0.0 once it is frozen
  SC_N = 24
};

struct Field64 {  // FP64 full field: two parities of double2 [12][sv]
  double2* p = nullptr;
};

}  // namespace qxd

// device work buffers owned by a lattice (allocated on first use, grown on demand): slots 0..28 the
// single-RHS solvers, 24..27 API staging, 29 and 31 FGCR vectors (31 also the training set), 30 the
// clover singular flag, 32..38 multi-RHS, 39 network application, 40 FGCR coefficients, 60 and 61
// the FP32 multi-RHS hop's tile records and its error word, 62 and 63 the clover build's scratch
#define QXD_WORK_SLOTS 64
struct qxd_lattice {
  qxd::Geom g;
  // device state of qxd_solve_batch when this lattice leads a batch (freed with the lattice)
  void* batch = nullptr;
  void (*batch_release)(void*) = nullptr;
  // deflation subspace and little Dirac operator (qxd_dfl_setup; freed with the lattice)
  void* dfl = nullptr;
  void (*dfl_release)(void*) = nullptr;
  // level 2 of the multigrid on top of it (qxd_mg_setup; freed with the lattice)
  void* mg = nullptr;
  void (*mg_release)(void*) = nullptr;
  qxd::i64 epoch = 0;  // counts changes of the gauge field or the clover term
  qxd::i64 mrt_epoch = -1;  // epoch of the multi-RHS hop's tile records (work slot 60)
  int Lphys[4];
  int tbc, cstar, order;
  qxd::i64 V, Vh, sv, Vphys;
  cudaStream_t stream = nullptr;
  int device = 0;

  // gauge field (FP64): SU(3) links, U(1) angles, hop links W = exp(iqA) U
  float4* U = nullptr;    // [2][4][9][sv] SU(3) links as double-float {re.hi, re.lo, im.hi, im.lo} (clover build)
  double* A = nullptr;    // [2][4][sv]
  double2* W64 = nullptr; // [2][4][9][sv]
  float2* W32 = nullptr;
  uint32_t* W16 = nullptr;   // FP16 pairs
  uint32_t* WB16 = nullptr;  // BF16 pairs
  double q = 0;
  bool have_gauge = false;

  // clover A (both parities) and inverse (index [parity]; filled on odd sites)
  double2* C64 = nullptr;  // [2][2][18][sv]
  double2* Ci64 = nullptr;
  float4* C32 = nullptr;   // [2][2][9][sv]
  float4* Ci32 = nullptr;
  uint2* C16 = nullptr;    // [2][2][9][sv]
  uint2* Ci16 = nullptr;
  float* C16n = nullptr;   // [2][2][sv]
  float* Ci16n = nullptr;
  uint2* CB16 = nullptr;
  uint2* CiB16 = nullptr;
  float* CB16n = nullptr;
  float* CiB16n = nullptr;
  bool have_clover = false;
  double m0 = 0, csw = 0, csw_qed = 0;

  // reductions: per-block partials, a ticket counter, device scalars, pinned host mirror
  double* red = nullptr;
  unsigned int* ticket = nullptr;
  double* scal = nullptr;
  double* hscal = nullptr;
  int red_blocks = 0;
  // multi-RHS reduction state (allocated on first use): per-RHS partials, tickets, scalars
  double* mr_red = nullptr;
  unsigned int* mr_ticket = nullptr;
  double* mr_scal = nullptr;
  double* mr_hscal = nullptr;
  int mr_cap = 0;

  // staging buffer for host/device boundary arrays
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // work buffers (lazily allocated): slots 0..23 and 28 solver, 24..27 API staging fields, 30 clover flag,
  // 32..39 multi-RHS fields
  void* work[QXD_WORK_SLOTS] = {nullptr};
  size_t work_bytes[QXD_WORK_SLOTS] = {0};

  // profiling
  bool profiling = false;
  qxd::i64 kcount[qxd::KSTAT_N] = {0};
  double kms[qxd::KSTAT_N] = {0};
  double kbytes[qxd::KSTAT_N] = {0};
  std::vector<cudaEvent_t> ev_pool;  // pairs (begin, end) per timed launch, reused after a flush
  std::vector<int> ev_kind;
  std::vector<double> ev_bytes;
  int ev_used = 0;
  qxd::i64 launches = 0;

  std::string err;
};

namespace qxd {

// Record an error message and return the status.
qxd_status fail(qxd_lattice* lat, qxd_status st, const std::string& msg);
qxd_status cuda_fail(qxd_lattice* lat, cudaError_t e, const char* where);

#define QXD_CUDA(lat, call)                                   \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return qxd::cuda_fail(lat, _e, #call); \
  } while (0)

#define QXD_CHECK_LAUNCH(lat, name)                                \
  do {                                                             \
    cudaError_t _e = cudaGetLastError();                           \
    if (_e != cudaSuccess) return qxd::cuda_fail(lat, _e, name);   \
    (lat)->launches++;                                             \
  } while (0)

// A vector argument that kernels read or write directly: it must be memory the current device
// can address (device or managed memory, not a plain host pointer) and start on an `align`-byte
// boundary (kernels move it in 8- or 16-byte words).  QXD_EINVAL otherwise, so that a host
// array or an offset view is refused on the host instead of faulting on the GPU.
qxd_status check_device_vector(qxd_lattice* lat, const void* p, size_t align, const char* what);

qxd_status ensure_work(qxd_lattice* lat, int slot, size_t bytes, void** out);
qxd_status ensure_stage(qxd_lattice* lat, size_t bytes);

inline int grid_for(i64 n, int bs) { return (int)((n + bs - 1) / bs); }

// ---- layout.cu ----
qxd_status pack_spinor64(qxd_lattice* lat, const double2* bnd, double2* field, int nsites_half_only);
qxd_status unpack_spinor64(qxd_lattice* lat, const double2* field, double2* bnd, int nsites_half_only);
qxd_status ingest_gauge(qxd_lattice* lat, const double2* su3, const double* a);
qxd_status ingest_gauge_openqxd(qxd_lattice* lat, const double2* u8, const double* a8);
qxd_status convert_links_low(qxd_lattice* lat);
qxd_status f64_to_f32(qxd_lattice* lat, const double2* in, float4* out, i64 nplanes_sites);
qxd_status f32_to_f64(qxd_lattice* lat, const float4* in, double2* out, i64 nplanes_sites);
qxd_status f32_to_n16(qxd_lattice* lat, const float4* in, uint2* out, float* nrm, int bf16);
qxd_status n16_to_f32(qxd_lattice* lat, const uint2* in, const float* nrm, float4* out, int bf16);

// ---- clover.cu ----
qxd_status clover_build(qxd_lattice* lat);
qxd_status clover_rebuild_sites(qxd_lattice* lat, const uint32_t* list, i64 nl, double* Fc, int* bad);
// link update on the device (layout.cu): scatter, re-derive W, mark the clover sites it touches
qxd_status update_links(qxd_lattice* lat, i64 n, const int64_t* idx, const double2* su3, const double* a,
                        unsigned char* mask, int* bad);
qxd_status compact_mask(qxd_lattice* lat, const unsigned char* mask, uint32_t* list, unsigned int* count);
qxd_status clover_export(qxd_lattice* lat, double* bnd);
// out = C in on one parity (site-local); which = 0 clover, 1 inverse
qxd_status clover_apply64(qxd_lattice* lat, int par, int which, const double2* in, double2* out);
qxd_status clover_apply32(qxd_lattice* lat, int par, int which, const float4* in, float4* out);

// ---- dslash.cu ----
enum Epi { EPI_HOP = 0, EPI_DFULL = 1, EPI_INV = 2, EPI_DHAT2 = 3, EPI_XPAY = 4, EPI_INVXPAY = 5 };
// One hop kernel launch for output parity `par`:
//   in   : spinor field of parity 1-par (neighbours)
//   same : spinor field of parity par (diagonal term), may be null for EPI_HOP/EPI_INV
//   out  : spinor field of parity par
// Epilogues:  HOP: out = coef H in;  DFULL: out = A same - 1/2 H in;
//             INV: out = A^-1 (coef H g5? in);  DHAT2: out = A same + coef g5? H in;
//             XPAY: out = same + coef H in;  INVXPAY: out = A^-1 (same + coef H in).
// g5 = 1 applies gamma5 to the neighbours (INV) or to the hop sum (DHAT2).
qxd_status hop64(qxd_lattice* lat, int par, int epi, int g5, const double2* in, const double2* same,
                 double2* out, double coef);
qxd_status hop32(qxd_lattice* lat, int par, int epi, int g5, const float4* in, const float4* same,
                 float4* out, float coef);
// 16-bit operator: spinors with per-site norms; output 16-bit (out_nrm != null) or FP32 (out32)
qxd_status hop16(qxd_lattice* lat, int bf16, int par, int epi, int g5, const uint2* in, const float* in_nrm,
                 const uint2* same, const float* same_nrm, uint2* out, float* out_nrm, float4* out32,
                 float coef);

// ---- mrhs.cu: FP32 hop on nrhs right-hand sides (fields at base + r * rs float4s) ----
// 16-bit multi-RHS hop: right-hand side r of a 16-bit field at base + r * 6 sv (uint2) with its
// norms at base + r * sv; FP32 output (out32, RHS r at + r * 6 sv float4s) or 16-bit output.
qxd_status hop16_mrhs(qxd_lattice* lat, int bf16, int par, int epi, int g5, const uint2* in, const float* in_nrm,
                      const uint2* same, const float* same_nrm, uint2* out, float* out_nrm, float4* out32, float coef,
                      int nrhs);
// nrhs right-hand sides at base + r * rs; rhs (host array of nrhs indices, or null for 0..nrhs-1)
// selects which ones
qxd_status hop32_mrhs(qxd_lattice* lat, int par, int epi, int g5, const float4* in, const float4* same, float4* out,
                      float coef, int nrhs, i64 rs, const int* rhs = nullptr);
// QXD_ETIMEOUT if a bounded wait of the FP32 multi-RHS hop expired since its records were built
// (synchronises the stream)
qxd_status mrhs_tile_status(qxd_lattice* lat);

// ---- blas.cu ----
// n = number of complex entries; arrays are double2 (FP64) or float2-pairs (FP32 as float4 * n/2)
qxd_status blas_norm2_64(qxd_lattice* lat, const double2* a, i64 n, int slot);
qxd_status blas_dot_64(qxd_lattice* lat, const double2* a, const double2* b, i64 n, int slot_re);
qxd_status blas_axpy_64(qxd_lattice* lat, double re, double im, const double2* x, double2* y, i64 n);
qxd_status blas_xpay_64(qxd_lattice* lat, const double2* x, double a, double2* y, i64 n);  // y = x + a y
qxd_status blas_copy(qxd_lattice* lat, void* dst, const void* src, size_t bytes);
qxd_status blas_zero(qxd_lattice* lat, void* dst, size_t bytes);
qxd_status blas_norm2_32(qxd_lattice* lat, const float4* a, i64 n4, int slot);
// CG (CGLS) fused updates; alpha = scal[SC_GAMMA] / scal[SC_QQ]
//   x += alpha p; s -= alpha q; scal[SC_SS] = ||s||^2
qxd_status cg_update_xs_64(qxd_lattice* lat, double2* x, const double2* p, double2* s, const double2* q, i64 n);
// (one thread per site; s16/p16 non-null also writes the 16-bit copy with its per-site scale)
qxd_status cg_update_xs_32(qxd_lattice* lat, float4* x, const float4* p, float4* s, const float4* q, uint2* s16,
                           float* s16n, int bf16);
//   p = r + (scal[SC_GAMMA_NEW] / scal[SC_GAMMA]) p; then scal[SC_GAMMA] = scal[SC_GAMMA_NEW]
qxd_status cg_update_p_64(qxd_lattice* lat, const double2* r, double2* p, i64 n);
qxd_status cg_update_p_32(qxd_lattice* lat, const float4* r, float4* p, uint2* p16, float* p16n, int bf16);
qxd_status cg_update_xs_32_full(qxd_lattice* lat, float4* x, const float4* p, float4* s, const float4* q);
qxd_status cg_update_p_32_full(qxd_lattice* lat, const float4* r, float4* p);
qxd_status read_scalars(qxd_lattice* lat, int first, int count, double* out);
qxd_status set_scalar(qxd_lattice* lat, int slot, double v);
// y += x (FP32 x widened into FP64 y), n = complex entries of y
qxd_status blas_acc_f32_into_f64(qxd_lattice* lat, const float4* x, double2* y, i64 n4);
qxd_status blas_axpy_32(qxd_lattice* lat, float a, const float4* x, float4* y, i64 n4);

// ---- bicgstab.cu (FP32 vectors, one thread per site; 16-bit copies written when non-null) ----
// Reduction state the BiCGStab kernels use: the lattice's own (single RHS), or the multi-RHS
// buffers starting at right-hand side r0 (mr = true).  nrhs consecutive right-hand sides run
// in one launch; RHS r's vectors sit at base + r * rs float4s.
struct Rhs {
  int nrhs = 1;
  i64 rs = 0;
  bool mr = false;
  int r0 = 0;
};
qxd_status bicg_cdot(qxd_lattice* lat, const float4* a, const float4* b, int slot, Rhs R = Rhs());
qxd_status bicg_s(qxd_lattice* lat, const float4* r, const float4* v, float4* s, uint2* s16, float* s16n, int bf16,
                  Rhs R = Rhs());
qxd_status bicg_ts(qxd_lattice* lat, const float4* t, const float4* s, Rhs R = Rhs());
qxd_status bicg_xr(qxd_lattice* lat, float4* x, const float4* p, const float4* s, const float4* t, const float4* rh,
                   float4* r, Rhs R = Rhs());
qxd_status bicg_p(qxd_lattice* lat, const float4* r, const float4* v, float4* p, uint2* p16, float* p16n, int bf16,
                  Rhs R = Rhs());
// device scalar write anywhere in the scalar arrays
qxd_status set_scalar_at(qxd_lattice* lat, double* p, double v);
// multi-RHS reduction state for up to n right-hand sides
qxd_status ensure_mrhs(qxd_lattice* lat, int n);
qxd_status bicg_copy(qxd_lattice* lat, const float4* r, float4* p, uint2* p16, float* p16n, int bf16);

// ---- profiling helpers (api.cu) ----
void prof_begin(qxd_lattice* lat, int kind, double bytes);
void prof_end(qxd_lattice* lat);
void prof_set_last_bytes(qxd_lattice* lat, double bytes);  // bytes of the last timed launch, known after it ran

// ---- solver.cu ----
qxd_status solve(qxd_lattice* lat, double2* x_field, const double2* b_field, const qxd_solve_params* p,
                 qxd_solve_info* info);
// full D on FP64 fields (both parities): out = D in
qxd_status apply_D64(qxd_lattice* lat, const double2* in, double2* out);
// ---- ptc.cu ----
qxd_status net_apply32(qxd_net* net, const float4* in, float4* out);  // full FP32 fields
qxd_status net_apply_adj32(qxd_net* net, const float4* in, float4* out);  // the adjoint network M^+
qxd_status net_check(qxd_net* net);  // error word of the tensor-core layers (synchronises)
size_t ptc_tc_packed_bytes(int cin, int cout);
qxd_status ptc_pack_weights(qxd_lattice* lat, int cin, int cout, const float2* Om, void* Bp);
size_t ptc_tc_pull_scratch(int cin, int cout, i64 sv);  // float4s of the pull form's virtual channels
qxd_status ptc_layer_tc(qxd_lattice* lat, int cin, int cout, const void* in, int in16, const void* Bp, void* out,
                        int out16, void* scratch, int* err);
// ---- solver_mrhs.cu ----
qxd_status solve_mrhs(qxd_lattice* lat, double2* x, const double2* b, int n, const qxd_solve_params* p,
                      qxd_solve_info* info);

}  // namespace qxd
