// Double-float arithmetic for the FP64 parts that are products of link matrices.
//
// FP64 runs at 1/64 of the FP32 rate on GB300, so the clover field strength (3x3 complex
// products of SU(3) links, eight per site and plane) is computed with double-float numbers: a
// value is hi + lo with two floats, |lo| <= ulp(hi) / 2, 48 significant bits (relative rounding
// 2^-47 against 2^-53 for FP64).  The building blocks are the error-free transformations of
// floating-point arithmetic: Knuth's TwoSum (a + b = s + e exactly, six additions) and the
// product with a fused multiply-add (a b = p + e exactly, e = fma(a, b, -p)).  A sum of products
// is accumulated as in the compensated dot product of Ogita, Rump and Oishi ("Accurate sum and
// dot product", SIAM J. Sci. Comput. 26, 2005): the leading float sum and the exact rounding
// errors of every step are kept apart and added once at the end.  The intrinsics __fadd_rn,
// __fmul_rn and __fmaf_rn keep the compiler from contracting or reassociating these steps.
#pragma once

#include <cstdint>

namespace qxd {

struct df {
  float hi, lo;
};

// x = hi + lo with hi = x rounded to float and lo = the remainder rounded to float
__device__ __forceinline__ df df_split(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double df_join(df a) { return (double)a.hi + (double)a.lo; }

// s + c: running sum of products; s is the leading float sum, c collects the low-order parts
struct dacc {
  float s, c;
};

__device__ __forceinline__ dacc dacc_zero() { return {0.f, 0.f}; }

// a += (xh + xl)(yh + yl), dropping xl yl (below 2^-48 of the product)
__device__ __forceinline__ void dacc_mac(dacc& a, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  float e = __fmaf_rn(xh, yh, -p);  // xh yh = p + e exactly
  e = __fmaf_rn(xh, yl, e);
  e = __fmaf_rn(xl, yh, e);
  const float s = __fadd_rn(a.s, p);  // TwoSum(a.s, p) = s + t
  const float bv = __fsub_rn(s, a.s);
  const float t = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bv)), __fsub_rn(p, bv));
  a.s = s;
  a.c = __fadd_rn(a.c, __fadd_rn(t, e));
}

// the accumulated value as a normalised double-float (TwoSum of s and c)
__device__ __forceinline__ df dacc_get(const dacc& a) {
  const float h = __fadd_rn(a.s, a.c);
  const float bv = __fsub_rn(h, a.s);
  const float l = __fadd_rn(__fsub_rn(a.s, __fsub_rn(h, bv)), __fsub_rn(a.c, bv));
  return {h, l};
}

// Complex double-float 3x3 matrices (row-major).
struct cdf {
  df re, im;
};
struct M3d {
  cdf m[9];
};

// acc[2 k] (re) and acc[2 k + 1] (im) += (a b)_k, with optional daggers on a and / or b
template <bool DA, bool DB>
__device__ __forceinline__ void mac3(dacc acc[18], const M3d& a, const M3d& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const cdf x = DA ? a.m[3 * k + i] : a.m[3 * i + k];
        const cdf y = DB ? b.m[3 * j + k] : b.m[3 * k + j];
        const float sx = DA ? -1.f : 1.f, sy = DB ? -1.f : 1.f;  // conjugation flips the imaginary parts
        const float xih = sx * x.im.hi, xil = sx * x.im.lo, yih = sy * y.im.hi, yil = sy * y.im.lo;
        dacc& re = acc[2 * (3 * i + j)];
        dacc& im = acc[2 * (3 * i + j) + 1];
        dacc_mac(re, x.re.hi, x.re.lo, y.re.hi, y.re.lo);
        dacc_mac(re, -xih, -xil, yih, yil);
        dacc_mac(im, x.re.hi, x.re.lo, yih, yil);
        dacc_mac(im, xih, xil, y.re.hi, y.re.lo);
      }
}

__device__ __forceinline__ M3d dacc_m3(const dacc acc[18]) {
  M3d r;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    r.m[k].re = dacc_get(acc[2 * k]);
    r.m[k].im = dacc_get(acc[2 * k + 1]);
  }
  return r;
}

template <bool DA, bool DB>
__device__ __forceinline__ M3d mul_d(const M3d& a, const M3d& b) {
  dacc acc[18];
#pragma unroll
  for (int k = 0; k < 18; ++k) acc[k] = dacc_zero();
  mac3<DA, DB>(acc, a, b);
  return dacc_m3(acc);
}

// a complex double-float stored as float4 {re.hi, re.lo, im.hi, im.lo}
__device__ __forceinline__ cdf cdf_load(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 cdf_store(const cdf& c) { return make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo); }
__device__ __forceinline__ float4 cdf_split(double re, double im) {
  const df r = df_split(re), i = df_split(im);
  return make_float4(r.hi, r.lo, i.hi, i.lo);
}

}  // namespace qxd
