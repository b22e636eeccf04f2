// Spin projection, link transport and reconstruction of one hop, shared by the single- and
// multi-right-hand-side hop kernels.
//
// Chiral basis (gamma_0 = [[0,-1],[-1,0]], gamma_k = [[0,-i s_k],[i s_k,0]]):
//   (1 -+ gamma_0) psi = [h; +-h]        with h = up +- dn
//   (1 -+ gamma_k) psi = [h; -+ i s_k h] with h = up +- i s_k dn
// (up = spins 0,1; dn = spins 2,3): each hop moves a 2-spin x 3-colour half spinor through one
// 3x3 link multiply.
#pragma once

#include "qxd_internal.cuh"

namespace qxd {

template <typename R, int MU, bool FWD>
__device__ __forceinline__ void project(const cplx<R> s[12], cplx<R> h[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cplx<R> up0 = s[c], up1 = s[3 + c], dn0 = s[6 + c], dn1 = s[9 + c];
    if (MU == 0) {
      h[c] = FWD ? up0 + dn0 : up0 - dn0;
      h[3 + c] = FWD ? up1 + dn1 : up1 - dn1;
    } else if (MU == 1) {  // i s_1 dn = (i dn1, i dn0)
      h[c] = FWD ? up0 + timesI(dn1) : up0 - timesI(dn1);
      h[3 + c] = FWD ? up1 + timesI(dn0) : up1 - timesI(dn0);
    } else if (MU == 2) {  // i s_2 dn = (dn1, -dn0)
      h[c] = FWD ? up0 + dn1 : up0 - dn1;
      h[3 + c] = FWD ? up1 - dn0 : up1 + dn0;
    } else {  // i s_3 dn = (i dn0, -i dn1)
      h[c] = FWD ? up0 + timesI(dn0) : up0 - timesI(dn0);
      h[3 + c] = FWD ? up1 - timesI(dn1) : up1 + timesI(dn1);
    }
  }
}

// acc += (1 -+ gamma_mu) reconstructed from the transported half spinor g
template <typename R, int MU, bool FWD>
__device__ __forceinline__ void accumulate(cplx<R> acc[12], const cplx<R> g[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cplx<R> g0 = g[c], g1 = g[3 + c];
    acc[c] = acc[c] + g0;
    acc[3 + c] = acc[3 + c] + g1;
    if (MU == 0) {
      acc[6 + c] = FWD ? acc[6 + c] + g0 : acc[6 + c] - g0;
      acc[9 + c] = FWD ? acc[9 + c] + g1 : acc[9 + c] - g1;
    } else if (MU == 1) {  // -i s_1 g = (-i g1, -i g0)
      acc[6 + c] = FWD ? acc[6 + c] - timesI(g1) : acc[6 + c] + timesI(g1);
      acc[9 + c] = FWD ? acc[9 + c] - timesI(g0) : acc[9 + c] + timesI(g0);
    } else if (MU == 2) {  // -i s_2 g = (-g1, g0)
      acc[6 + c] = FWD ? acc[6 + c] - g1 : acc[6 + c] + g1;
      acc[9 + c] = FWD ? acc[9 + c] + g0 : acc[9 + c] - g0;
    } else {  // -i s_3 g = (-i g0, i g1)
      acc[6 + c] = FWD ? acc[6 + c] - timesI(g0) : acc[6 + c] + timesI(g0);
      acc[9 + c] = FWD ? acc[9 + c] + timesI(g1) : acc[9 + c] - timesI(g1);
    }
  }
}

// acc += sc (1 -+ gamma_mu) g: the same reconstruction with the half spinor's real scale (the per-site
// norm of a 16-bit neighbour spinor and the time-boundary sign) folded into fused multiply-adds
template <typename R, int MU, bool FWD>
__device__ __forceinline__ void accumulate_s(cplx<R> acc[12], const cplx<R> g[6], R sc) {
  auto add = [&](cplx<R>& a, cplx<R> b, R f) { a = mk(fma(f, b.re, a.re), fma(f, b.im, a.im)); };
  auto addi = [&](cplx<R>& a, cplx<R> b, R f) { a = mk(fma(-f, b.im, a.re), fma(f, b.re, a.im)); };  // a += f i b
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cplx<R> g0 = g[c], g1 = g[3 + c];
    add(acc[c], g0, sc);
    add(acc[3 + c], g1, sc);
    if (MU == 0) {
      add(acc[6 + c], g0, FWD ? sc : -sc);
      add(acc[9 + c], g1, FWD ? sc : -sc);
    } else if (MU == 1) {  // -i s_1 g = (-i g1, -i g0)
      addi(acc[6 + c], g1, FWD ? -sc : sc);
      addi(acc[9 + c], g0, FWD ? -sc : sc);
    } else if (MU == 2) {  // -i s_2 g = (-g1, g0)
      add(acc[6 + c], g1, FWD ? -sc : sc);
      add(acc[9 + c], g0, FWD ? sc : -sc);
    } else {  // -i s_3 g = (-i g0, i g1)
      addi(acc[6 + c], g0, FWD ? -sc : sc);
      addi(acc[9 + c], g1, FWD ? sc : -sc);
    }
  }
}

template <typename R, bool DAG>
__device__ __forceinline__ void link_mul(const cplx<R> u[9], const cplx<R> h[6], cplx<R> g[6]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cplx<R> r = DAG ? cjmul(u[a], h[3 * s]) : cmul(u[3 * a], h[3 * s]);
#pragma unroll
      for (int b = 1; b < 3; ++b) r = DAG ? cjmac(r, u[3 * b + a], h[3 * s + b]) : cmac(r, u[3 * a + b], h[3 * s + b]);
      g[3 * s + a] = r;
    }
}

}  // namespace qxd
