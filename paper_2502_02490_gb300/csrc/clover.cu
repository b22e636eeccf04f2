// Clover term on the GPU (Sec. 2: two Hermitian 6x6 chirality blocks per site; Sec. 4.1.3:
// 36-real packing; Sec. 4.3: QED clover term added to the SU(3) one; Sec. 6: generate the
// clover field on the GPU instead of uploading it).
//
// A(x) = (4 + m0) + c_sw (i/4) sum_{mu != nu} sigma_{mu nu} Fhat_{mu nu}
//                 + q c_sw^QED (i/4) sum_{mu != nu} sigma_{mu nu} fhat_{mu nu}
// with Fhat = (Q_{mu nu} - Q_{mu nu}^dag)/8 made traceless (Q = sum of the four plaquette
// leaves at x) and fhat = (i/4) sum_leaves sin(phi_leaf) from the U(1) angles.
//
// In the chiral basis sigma_{0k} = diag(s_k, -s_k) and sigma_{jk} = -eps_{jkl} diag(s_l, s_l)
// (s = Pauli matrices), so with G^{+-}_l = F_{0l} -+ Ftilde_l (Ftilde_1 = F_23, Ftilde_2 = F_31,
// Ftilde_3 = F_12):
//   A_+ = (4 + m0) + (i/2) sum_l s_l (x) [c_sw G^+_l + q c_sw^QED g^+_l]
//   A_- = (4 + m0) - (i/2) sum_l s_l (x) [c_sw G^-_l + q c_sw^QED g^-_l]
// and s_l (x) Y = [[Y_3, Y_1 - i Y_2], [Y_1 + i Y_2, -Y_3]] in the index 3*alpha' + a.
#include "df64.cuh"
#include "qxd_internal.cuh"

// minimum resident blocks per SM of the double-float product kernels (register budget)
#ifndef QXD_CLOVER_MINB
#define QXD_CLOVER_MINB 3
#endif

namespace qxd {

typedef cplx<double> cd;

struct M3 {
  cd m[9];
};

__device__ __forceinline__ void step(const Geom& g, int y[4], int mu, int dir) {
  y[mu] += dir;
  bool crossed = false;
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
}

// SU(3) link U_mu(y) from the double-float copy of the field
__device__ __forceinline__ M3d load_u(const Geom& g, const float4* __restrict__ U, const int y[4], int mu) {
  i64 lam = lexi(g, y);
  int par = (y[0] + y[1] + y[2] + y[3]) & 1;
  const float4* b = U + (i64)((par * 4 + mu) * 9) * g.sv + (lam >> 1);
  M3d r;
#pragma unroll
  for (int k = 0; k < 9; ++k) r.m[k] = cdf_load(b[k * g.sv]);
  return r;
}

__device__ __forceinline__ double load_a(const Geom& g, const double* __restrict__ A, const int y[4], int mu) {
  i64 lam = lexi(g, y);
  int par = (y[0] + y[1] + y[2] + y[3]) & 1;
  return A[(i64)(par * 4 + mu) * g.sv + (lam >> 1)];
}

// Plaquette half-products of the plane (MU, NU) at every site y: A(y) = U_mu(y) U_nu(y+mu),
// B(y) = U_nu(y) U_mu(y+nu) (so the plaquette at y is A B^+), in double-float arithmetic, and
// the sine of the U(1) plaquette angle A_mu(y) + A_nu(y+mu) - A_mu(y+nu) - A_nu(y) in FP64.
// Stored [k][2 sv]: k < 9 A, 9 <= k < 18 B (double-float complex as float4), then the sines
// [2 sv] (doubles).
template <int MU, int NU>
__global__ void __launch_bounds__(128, QXD_CLOVER_MINB) k_clover_half(Geom g, const float4* __restrict__ U, const double* __restrict__ A,
                                                     float4* __restrict__ Hb) {
  const i64 n = 2 * g.Vh, st = 2 * g.sv;
  for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < n; e += (i64)gridDim.x * blockDim.x) {
    const int par = e >= g.Vh ? 1 : 0;
    const i64 cb = e - (i64)par * g.Vh;
    int y[4];
    cb_coords(g, cb, par, y);
    int ym[4] = {y[0], y[1], y[2], y[3]}, yn[4] = {y[0], y[1], y[2], y[3]};
    step(g, ym, MU, +1);
    step(g, yn, NU, +1);
    const i64 s0 = (i64)par * g.sv + cb;
    {
      const M3d a = mul_d<false, false>(load_u(g, U, y, MU), load_u(g, U, ym, NU));
#pragma unroll
      for (int k = 0; k < 9; ++k) Hb[k * st + s0] = cdf_store(a.m[k]);
    }
    {
      const M3d b = mul_d<false, false>(load_u(g, U, y, NU), load_u(g, U, yn, MU));
#pragma unroll
      for (int k = 0; k < 9; ++k) Hb[(9 + k) * st + s0] = cdf_store(b.m[k]);
    }
    ((double*)(Hb + 18 * st))[s0] =
        sin(load_a(g, A, y, MU) + load_a(g, A, ym, NU) - load_a(g, A, yn, MU) - load_a(g, A, y, NU));
  }
}

__device__ __forceinline__ M3d load_h(const float4* __restrict__ Hb, i64 st, i64 s, int which) {
  M3d r;
#pragma unroll
  for (int k = 0; k < 9; ++k) r.m[k] = cdf_load(Hb[(which * 9 + k) * st + s]);
  return r;
}

// the sum of leaves in FP64
__device__ __forceinline__ M3 q_of(const dacc acc[18]) {
  M3 Q;
#pragma unroll
  for (int k = 0; k < 9; ++k) Q.m[k] = mk(df_join(dacc_get(acc[2 * k])), df_join(dacc_get(acc[2 * k + 1])));
  return Q;
}

__device__ __forceinline__ i64 site_of(const Geom& g, const int y[4]) {
  const int par = (y[0] + y[1] + y[2] + y[3]) & 1;
  return (i64)par * g.sv + (lexi(g, y) >> 1);
}

// Fhat = (Q - Q^+)/8 made traceless, and fhat, stored as 10 doubles of stride st at o: Im F_00,
// Im F_11, Im F_22, (Re, Im) F_01, F_02, F_12 (the rest follows from anti-Hermiticity), fhat.
__device__ __forceinline__ void store_fs(const M3& Q, double f1, double* __restrict__ o, i64 st) {
  M3 F;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const cd a = Q.m[3 * i + j], b = Q.m[3 * j + i];
      F.m[3 * i + j] = mk((a.re - b.re) * 0.125, (a.im + b.im) * 0.125);
    }
  const double tr_im = (F.m[0].im + F.m[4].im + F.m[8].im) / 3.0;
  F.m[0].im -= tr_im;
  F.m[4].im -= tr_im;
  F.m[8].im -= tr_im;
  o[0 * st] = F.m[0].im;
  o[1 * st] = F.m[4].im;
  o[2 * st] = F.m[8].im;
  o[3 * st] = F.m[1].re;
  o[4 * st] = F.m[1].im;
  o[5 * st] = F.m[2].re;
  o[6 * st] = F.m[2].im;
  o[7 * st] = F.m[5].re;
  o[8 * st] = F.m[5].im;
  o[9 * st] = f1;
}

// The four leaves of the plane (MU, NU) at x from the half-products of the plaquettes around it:
//   leaf 1 = A(x) B(x)^+,  leaf 2 = U_nu(x) B(x-mu)^+ U_mu(x-mu),  leaf 3 = B(x-mu-nu)^+ A(x-mu-nu),
//   leaf 4 = U_nu(x-nu)^+ A(x-nu) U_mu(x)^+
// (each leaf is its plaquette rotated to start at x, so its U(1) angle is the plaquette's);
// then Fhat = (Q - Q^+)/8 traceless and fhat = 1/4 sum of the sines, stored in the compact layout below.
template <int MU, int NU>
__global__ void __launch_bounds__(128, QXD_CLOVER_MINB) k_clover_leaves(Geom g, const float4* __restrict__ U, const float4* __restrict__ Hb,
                                                       int p, double* __restrict__ Fb) {
  const i64 n = 2 * g.Vh, st = 2 * g.sv;
  const double* sn = (const double*)(Hb + 18 * st);
  for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < n; e += (i64)gridDim.x * blockDim.x) {
    const int par = e >= g.Vh ? 1 : 0;
    const i64 cb = e - (i64)par * g.Vh;
    int x[4];
    cb_coords(g, cb, par, x);
    int xm[4] = {x[0], x[1], x[2], x[3]}, xn[4] = {x[0], x[1], x[2], x[3]};
    step(g, xm, MU, -1);
    step(g, xn, NU, -1);
    int xmn[4] = {xm[0], xm[1], xm[2], xm[3]};
    step(g, xmn, NU, -1);
    const i64 s0 = (i64)par * g.sv + cb, s1 = site_of(g, xm), s2 = site_of(g, xmn), s3 = site_of(g, xn);
    // Q = the sum of the four leaves; the last product of every leaf accumulates into Q directly
    dacc q[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) q[k] = dacc_zero();
    mac3<false, true>(q, load_h(Hb, st, s0, 0), load_h(Hb, st, s0, 1));
    mac3<false, false>(q, mul_d<false, true>(load_u(g, U, x, NU), load_h(Hb, st, s1, 1)), load_u(g, U, xm, MU));
    mac3<true, false>(q, load_h(Hb, st, s2, 1), load_h(Hb, st, s2, 0));
    mac3<false, true>(q, mul_d<true, false>(load_u(g, U, xn, NU), load_h(Hb, st, s3, 0)), load_u(g, U, x, MU));
    store_fs(q_of(q), 0.25 * (sn[s0] + sn[s1] + sn[s2] + sn[s3]), Fb + (i64)p * 10 * st + s0, st);
  }
}

// The link-update path: the field strength of the plane (MU, NU) at listed sites only (list
// entries par * Vh + cb), each leaf multiplied out from the links (3 products per leaf) and the
// U(1) part from the four plaquette angles; written in the layout of k_clover_leaves at list
// position e with stride nl.
template <int MU, int NU>
__global__ void __launch_bounds__(128) k_fs_sites(Geom g, const float4* __restrict__ U, const double* __restrict__ A,
                                                  const uint32_t* __restrict__ list, i64 nl, int p,
                                                  double* __restrict__ Fc) {
  for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < nl; e += (i64)gridDim.x * blockDim.x) {
    const i64 t = list[e];
    const int par = t >= g.Vh ? 1 : 0;
    int x[4];
    cb_coords(g, t - (i64)par * g.Vh, par, x);
    int xpm[4] = {x[0], x[1], x[2], x[3]}, xpn[4] = {x[0], x[1], x[2], x[3]};
    int xm[4] = {x[0], x[1], x[2], x[3]}, xn[4] = {x[0], x[1], x[2], x[3]};
    step(g, xpm, MU, +1);
    step(g, xpn, NU, +1);
    step(g, xm, MU, -1);
    step(g, xn, NU, -1);
    int xmn[4] = {xm[0], xm[1], xm[2], xm[3]}, xmpn[4] = {xm[0], xm[1], xm[2], xm[3]};
    int xnpm[4] = {xn[0], xn[1], xn[2], xn[3]};
    step(g, xmn, NU, -1);
    step(g, xmpn, NU, +1);
    step(g, xnpm, MU, +1);
    dacc q[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) q[k] = dacc_zero();
    // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
    mac3<false, true>(q,
                      mul_d<false, true>(mul_d<false, false>(load_u(g, U, x, MU), load_u(g, U, xpm, NU)),
                                         load_u(g, U, xpn, MU)),
                      load_u(g, U, x, NU));
    // leaf 2: U_nu(x) U_mu(x-mu+nu)^+ U_nu(x-mu)^+ U_mu(x-mu)
    mac3<false, false>(q,
                       mul_d<false, true>(mul_d<false, true>(load_u(g, U, x, NU), load_u(g, U, xmpn, MU)),
                                          load_u(g, U, xm, NU)),
                       load_u(g, U, xm, MU));
    // leaf 3: U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
    mac3<false, false>(q,
                       mul_d<false, false>(mul_d<true, true>(load_u(g, U, xm, MU), load_u(g, U, xmn, NU)),
                                           load_u(g, U, xmn, MU)),
                       load_u(g, U, xn, NU));
    // leaf 4: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
    mac3<false, true>(q,
                      mul_d<false, false>(mul_d<true, false>(load_u(g, U, xn, NU), load_u(g, U, xn, MU)),
                                          load_u(g, U, xnpm, NU)),
                      load_u(g, U, x, MU));
    // U(1): plaquette angle th(c) = A_mu(c) + A_nu(c+mu) - A_mu(c+nu) - A_nu(c) at the corners
    // x, x-mu, x-mu-nu, x-nu of the four leaves
    const double s0 = sin(load_a(g, A, x, MU) + load_a(g, A, xpm, NU) - load_a(g, A, xpn, MU) - load_a(g, A, x, NU));
    const double s1 = sin(load_a(g, A, xm, MU) + load_a(g, A, x, NU) - load_a(g, A, xmpn, MU) - load_a(g, A, xm, NU));
    const double s2 = sin(load_a(g, A, xmn, MU) + load_a(g, A, xn, NU) - load_a(g, A, xm, MU) - load_a(g, A, xmn, NU));
    const double s3 = sin(load_a(g, A, xn, MU) + load_a(g, A, xnpm, NU) - load_a(g, A, x, MU) - load_a(g, A, xn, NU));
    store_fs(q_of(q), 0.25 * (s0 + s1 + s2 + s3), Fc + (i64)p * 10 * nl + e, nl);
  }
}

// Field strengths per site and plane (written by k_clover_leaves): planes 0..2 = (0,1) (0,2)
// (0,3), 3 = (2,3), 4 = (1,3), 5 = (1,2); 10 doubles [plane][k][2 sv]: Im F_00, Im F_11, Im F_22,
// (Re, Im) F_01, F_02, F_12 (the lower triangle is -conj), and fhat.
// Y_l = c_sw (F_el + smag F_ml) + i q c_sw^QED (f_el + smag f_ml) 1 (anti-Hermitian, 3x3), as a
// full 3x3 array (the lower triangle is -conj of the upper).
__device__ __forceinline__ void y_full(const double* __restrict__ Fb, i64 st, i64 s, int l, double smag, double csw,
                                       double cq, cd Y[9]) {
  const double* e = Fb + (i64)l * 10 * st + s;
  const double* m = Fb + (i64)(3 + l) * 10 * st + s;
  const double gv = cq * (e[9 * st] + smag * m[9 * st]);
  Y[0] = mk(0.0, csw * (e[0] + smag * m[0]) + gv);
  Y[4] = mk(0.0, csw * (e[st] + smag * m[st]) + gv);
  Y[8] = mk(0.0, csw * (e[2 * st] + smag * m[2 * st]) + gv);
  Y[1] = mk(csw * (e[3 * st] + smag * m[3 * st]), csw * (e[4 * st] + smag * m[4 * st]));
  Y[2] = mk(csw * (e[5 * st] + smag * m[5 * st]), csw * (e[6 * st] + smag * m[6 * st]));
  Y[5] = mk(csw * (e[7 * st] + smag * m[7 * st]), csw * (e[8 * st] + smag * m[8 * st]));
  Y[3] = mk(-Y[1].re, Y[1].im);
  Y[6] = mk(-Y[2].re, Y[2].im);
  Y[7] = mk(-Y[5].re, Y[5].im);
}

// A_+- of every site from the stored field strengths: G^{+-}_l = F_{0l} -+ sgn_l F_mag(l) with the
// magnetic planes (2,3), (1,3), (1,2) of sign +1, -1, +1; one chiral block at a time.  With
// s = side i (side = +1/2 on A_+, -1/2 on A_-) the block is diag 1 + s sum_l sigma_l (x) Y_l, i.e.
// in 3x3 spin blocks: upper left diag + s Y_3, lower right diag - s Y_3, upper right
// s Y_1 - i s Y_2 (the lower left is its adjoint).  Only the stored upper triangle is formed, so
// the block is Hermitian by construction.
// With a list (link-update path) only the listed sites, their field strengths at list position e
// with stride nl.
__global__ void __launch_bounds__(128) k_clover_assemble(Geom g, const double* __restrict__ Fb, double diag, double csw,
                                                         double cq, double2* __restrict__ C,
                                                         const uint32_t* __restrict__ list, i64 nl) {
  const i64 n = list ? nl : 2 * g.Vh, st = list ? nl : 2 * g.sv;
  for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < n; e += (i64)gridDim.x * blockDim.x) {
    const i64 t = list ? (i64)list[e] : e;
    const int par = t >= g.Vh ? 1 : 0;
    const i64 cb = t - (i64)par * g.Vh;
    const i64 s = list ? e : (i64)par * g.sv + cb;
#pragma unroll
    for (int blkid = 0; blkid < 2; ++blkid) {
      const double side = blkid == 0 ? 0.5 : -0.5;
      const double smag1 = blkid == 0 ? -1.0 : 1.0;  // smag_l = -+ sgn_l, sgn = (+1, -1, +1)
      cd y1[9], y2[9], y3[9];
      y_full(Fb, st, s, 0, smag1, csw, cq, y1);
      y_full(Fb, st, s, 1, -smag1, csw, cq, y2);
      y_full(Fb, st, s, 2, smag1, csw, cq, y3);
      // packed block: entries 0..2 the six real diagonal elements in pairs, 3 + k the k-th element
      // (i < j, row-major) of the upper triangle
      double2* out = C + (i64)((par * 2 + blkid) * 18) * g.sv + cb;
      // diagonal: diag -+ side Im Y_3,aa (Re of s Y_3,aa = -side Im Y_3,aa)
      out[0] = make_double2(diag - side * y3[0].im, diag - side * y3[4].im);
      out[g.sv] = make_double2(diag - side * y3[8].im, diag + side * y3[0].im);
      out[2 * g.sv] = make_double2(diag + side * y3[4].im, diag + side * y3[8].im);
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i + 1; j < 6; ++j) {
          const int k = i * 5 - i * (i - 1) / 2 + (j - i - 1);  // position of (i, j) in the upper triangle
          const int al = i / 3, a = i % 3, be = j / 3, b = j % 3;
          cd v;
          if (al == 0 && be == 0) {  // s Y_3
            const cd w = y3[3 * a + b];
            v = mk(-side * w.im, side * w.re);
          } else if (al == 1) {  // -s Y_3
            const cd w = y3[3 * a + b];
            v = mk(side * w.im, -side * w.re);
          } else {  // s Y_1 - i s Y_2 = side (i Y_1 + Y_2)
            const cd w1 = y1[3 * a + b], w2 = y2[3 * a + b];
            v = mk(side * (w2.re - w1.im), side * (w1.re + w2.im));
          }
          out[(3 + k) * g.sv] = make_double2(v.re, v.im);
        }
    }
  }
}

// One step (column C) of in-place Gauss-Jordan inversion with partial pivoting; C is a template
// argument so that every index is static and the block stays in registers.
template <int C>
__device__ __forceinline__ void gj_step(cd a[6][6], double amax, int piv[6], bool& singular) {
  int pc = C;
  double best = a[C][C].re * a[C][C].re + a[C][C].im * a[C][C].im;
#pragma unroll
  for (int i = C + 1; i < 6; ++i) {
    const double m = a[i][C].re * a[i][C].re + a[i][C].im * a[i][C].im;
    if (m > best) {
      best = m;
      pc = i;
    }
  }
  piv[C] = pc;
  if (!(sqrt(best) > 1e-14 * amax)) singular = true;  // strict: an all-zero block is singular
#pragma unroll
  for (int i = C + 1; i < 6; ++i) {
    const bool sw = pc == i;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const cd u = a[C][j], v = a[i][j];
      a[C][j] = sw ? v : u;
      a[i][j] = sw ? u : v;
    }
  }
  const cd p = a[C][C];
  const double pm = p.re * p.re + p.im * p.im;
  const cd pinv = pm > 0.0 ? mk(p.re / pm, -p.im / pm) : mk(0.0, 0.0);
  a[C][C] = mk(1.0, 0.0);
#pragma unroll
  for (int j = 0; j < 6; ++j) a[C][j] = cmul(a[C][j], pinv);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (i == C) continue;
    const cd f = a[i][C];
    a[i][C] = mk(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 6; ++j) a[i][j] = a[i][j] - cmul(f, a[C][j]);
  }
}

template <int C>
__device__ __forceinline__ void gj_unswap(cd a[6][6], const int piv[6]) {
#pragma unroll
  for (int j = C + 1; j < 6; ++j) {
    const bool sw = piv[C] == j;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const cd u = a[i][C], v = a[i][j];
      a[i][C] = sw ? v : u;
      a[i][j] = sw ? u : v;
    }
  }
}

// Inverse of each Hermitian 6x6 block of the odd sites by in-place Gauss-Jordan elimination with
// partial pivoting (FP64), fully unrolled so that the block stays in registers (row swaps are
// predicated; the row permutation is undone as column swaps at the end).  A block whose pivot
// falls below 1e-14 times its largest entry sets *bad.  Only the odd-site inverse is used
// (A_oo^-1 of the Schur complement and of the reconstruction).
// With a list (link-update path): the odd listed sites only.
__global__ void __launch_bounds__(128) k_clover_invert(Geom g, const double2* __restrict__ C,
                                                       double2* __restrict__ Ci, int* __restrict__ bad,
                                                       const uint32_t* __restrict__ list, i64 nl) {
  const i64 nsites = list ? nl : g.Vh;
  const i64 n = 2 * nsites;  // (odd site, block)
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int blkid = (int)(t / nsites);
    i64 cb = t - (i64)blkid * nsites;
    if (list) {
      const i64 v = list[cb];
      if (v < g.Vh) continue;  // even site: no inverse needed
      cb = v - g.Vh;
    }
    const double2* in = C + (i64)((2 + blkid) * 18) * g.sv + cb;
    // packed: pairs 0..2 the six real diagonal entries, pairs 3..17 the strict upper triangle
    cd a[6][6];
    double amax = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double2 v = in[k * g.sv];
      a[2 * k][2 * k] = mk(v.x, 0.0);
      a[2 * k + 1][2 * k + 1] = mk(v.y, 0.0);
      amax = fmax(amax, fmax(fabs(v.x), fabs(v.y)));
    }
    {
      int k = 3;
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i + 1; j < 6; ++j) {
          const double2 v = in[k * g.sv];
          a[i][j] = mk(v.x, v.y);
          a[j][i] = mk(v.x, -v.y);
          amax = fmax(amax, fabs(v.x) + fabs(v.y));
          ++k;
        }
    }
    bool singular = false;
    int piv[6];
    gj_step<0>(a, amax, piv, singular);
    gj_step<1>(a, amax, piv, singular);
    gj_step<2>(a, amax, piv, singular);
    gj_step<3>(a, amax, piv, singular);
    gj_step<4>(a, amax, piv, singular);
    gj_step<5>(a, amax, piv, singular);
    // undo the row interchanges as column interchanges, last first
    gj_unswap<5>(a, piv);
    gj_unswap<4>(a, piv);
    gj_unswap<3>(a, piv);
    gj_unswap<2>(a, piv);
    gj_unswap<1>(a, piv);
    gj_unswap<0>(a, piv);
    if (singular) atomicOr(bad, 1);
    double2* out = Ci + (i64)((2 + blkid) * 18) * g.sv + cb;
#pragma unroll
    for (int k = 0; k < 3; ++k) out[k * g.sv] = make_double2(a[2 * k][2 * k].re, a[2 * k + 1][2 * k + 1].re);
    {
      int k = 3;
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i + 1; j < 6; ++j) {
          // symmetrise the rounding of the two triangles
          out[k * g.sv] = make_double2(0.5 * (a[i][j].re + a[j][i].re), 0.5 * (a[i][j].im - a[j][i].im));
          ++k;
        }
    }
  }
}

// With a list (link-update path): the two blocks of each listed site.
__global__ void k_clover_low(Geom g, const double2* __restrict__ C, float4* __restrict__ C32,
                             uint2* __restrict__ C16, float* __restrict__ C16n, uint2* __restrict__ CB,
                             float* __restrict__ CBn, const uint32_t* __restrict__ list, i64 nl) {
  i64 n = list ? 2 * nl : 4 * g.sv;  // (parity, block, site incl. padding) or (listed site, block)
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    i64 pb, cb;
    if (list) {
      const i64 v = list[t >> 1];
      const int par = v >= g.Vh ? 1 : 0;
      pb = 2 * par + (t & 1);
      cb = v - (i64)par * g.Vh;
    } else {
      pb = t / g.sv;
      cb = t - pb * g.sv;
    }
    const double2* in = C + pb * 18 * g.sv + cb;
    float r[36];
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      double2 v = in[k * g.sv];
      r[2 * k] = (float)v.x;
      r[2 * k + 1] = (float)v.y;
      m = fmaxf(m, fmaxf(fabsf(r[2 * k]), fabsf(r[2 * k + 1])));
    }
    float inv = m > 0.f ? 1.f / m : 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      C32[(pb * 9 + k) * g.sv + cb] = make_float4(r[4 * k], r[4 * k + 1], r[4 * k + 2], r[4 * k + 3]);
      uint2 h, b;
      h.x = H16::pack(r[4 * k] * inv, r[4 * k + 1] * inv);
      h.y = H16::pack(r[4 * k + 2] * inv, r[4 * k + 3] * inv);
      b.x = B16::pack(r[4 * k] * inv, r[4 * k + 1] * inv);
      b.y = B16::pack(r[4 * k + 2] * inv, r[4 * k + 3] * inv);
      C16[(pb * 9 + k) * g.sv + cb] = h;
      CB[(pb * 9 + k) * g.sv + cb] = b;
    }
    C16n[pb * g.sv + cb] = m;
    CBn[pb * g.sv + cb] = m;
  }
}

static int grid_cap(i64 n, int bs) {
  i64 b = (n + bs - 1) / bs;
  return (int)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}

qxd_status clover_build(qxd_lattice* lat) {
  const Geom& g = lat->g;
  // field strengths of the six planes (one thread per site and plane), then the blocks; plane by
  // plane: plaquette half-products (and U(1) sines) at every site, then the four leaves of every
  // site from them (8 3x3 products per site and plane instead of 12).  Both scratch buffers
  // (field strengths: 10 doubles per site and plane; half-products: 19 x 16 B per site) stay
  // with the lattice (work slots 62 and 63), so a rebuild allocates nothing.
  double* Fb;
  float4* Hb;
  {
    void *f, *h;
    qxd_status st = ensure_work(lat, 62, sizeof(double) * 6 * 10 * 2 * g.sv, &f);
    if (st != QXD_OK) return st;
    st = ensure_work(lat, 63, sizeof(float4) * 19 * 2 * g.sv, &h);
    if (st != QXD_OK) return st;
    Fb = (double*)f;
    Hb = (float4*)h;
  }
  const int gc = grid_cap(2 * g.Vh, 128);
#define QXD_PLANE(P, M, N)                                                     \
  k_clover_half<M, N><<<gc, 128, 0, lat->stream>>>(g, lat->U, lat->A, Hb);      \
  QXD_CHECK_LAUNCH(lat, "k_clover_half");                                       \
  k_clover_leaves<M, N><<<gc, 128, 0, lat->stream>>>(g, lat->U, Hb, P, Fb);     \
  QXD_CHECK_LAUNCH(lat, "k_clover_leaves");
  QXD_PLANE(0, 0, 1)
  QXD_PLANE(1, 0, 2)
  QXD_PLANE(2, 0, 3)
  QXD_PLANE(3, 2, 3)
  QXD_PLANE(4, 1, 3)
  QXD_PLANE(5, 1, 2)
#undef QXD_PLANE
  k_clover_assemble<<<grid_cap(2 * g.Vh, 128), 128, 0, lat->stream>>>(g, Fb, 4.0 + lat->m0, lat->csw,
                                                                      lat->q * lat->csw_qed, lat->C64, nullptr, 0);
  QXD_CHECK_LAUNCH(lat, "k_clover_assemble");
  void* w;
  qxd_status st = ensure_work(lat, 30, sizeof(int), &w);  // slot 30: clover singular flag
  if (st) return st;
  int* bad = (int*)w;
  QXD_CUDA(lat, cudaMemsetAsync(bad, 0, sizeof(int), lat->stream));
  k_clover_invert<<<grid_cap(2 * g.Vh, 128), 128, 0, lat->stream>>>(g, lat->C64, lat->Ci64, bad, nullptr, 0);
  QXD_CHECK_LAUNCH(lat, "k_clover_invert");
  k_clover_low<<<grid_cap(4 * g.sv, 128), 128, 0, lat->stream>>>(g, lat->C64, lat->C32, lat->C16, lat->C16n,
                                                                 lat->CB16, lat->CB16n, nullptr, 0);
  QXD_CHECK_LAUNCH(lat, "k_clover_low");
  k_clover_low<<<grid_cap(4 * g.sv, 128), 128, 0, lat->stream>>>(g, lat->Ci64, lat->Ci32, lat->Ci16, lat->Ci16n,
                                                                 lat->CiB16, lat->CiB16n, nullptr, 0);
  QXD_CHECK_LAUNCH(lat, "k_clover_low");
  int hbad = 0;
  QXD_CUDA(lat, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, lat->stream));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  if (hbad) return fail(lat, QXD_ESINGULAR, "a clover block on an odd site is not invertible");
  return QXD_OK;
}

// Rebuild the clover blocks (A, the odd-site inverse and the FP32 / 16-bit copies) at the nl
// listed sites only (list entries par * Vh + cb, on the device), after a link update changed the
// plaquettes around them.  Same arithmetic as clover_build, with each leaf multiplied out from the
// links (12 products per site and plane) since the listed sites share no half-products.
qxd_status clover_rebuild_sites(qxd_lattice* lat, const uint32_t* list, i64 nl, double* Fc, int* bad) {
  const Geom& g = lat->g;
  if (nl <= 0) return QXD_OK;
  const int gc = grid_cap(nl, 128);
#define QXD_PLANE_SITES(P, M, N)                                                                \
  k_fs_sites<M, N><<<gc, 128, 0, lat->stream>>>(g, lat->U, lat->A, list, nl, P, Fc);            \
  QXD_CHECK_LAUNCH(lat, "k_fs_sites");
  QXD_PLANE_SITES(0, 0, 1)
  QXD_PLANE_SITES(1, 0, 2)
  QXD_PLANE_SITES(2, 0, 3)
  QXD_PLANE_SITES(3, 2, 3)
  QXD_PLANE_SITES(4, 1, 3)
  QXD_PLANE_SITES(5, 1, 2)
#undef QXD_PLANE_SITES
  k_clover_assemble<<<gc, 128, 0, lat->stream>>>(g, Fc, 4.0 + lat->m0, lat->csw, lat->q * lat->csw_qed, lat->C64,
                                                 list, nl);
  QXD_CHECK_LAUNCH(lat, "k_clover_assemble");
  k_clover_invert<<<grid_cap(2 * nl, 128), 128, 0, lat->stream>>>(g, lat->C64, lat->Ci64, bad, list, nl);
  QXD_CHECK_LAUNCH(lat, "k_clover_invert");
  k_clover_low<<<grid_cap(2 * nl, 128), 128, 0, lat->stream>>>(g, lat->C64, lat->C32, lat->C16, lat->C16n, lat->CB16,
                                                               lat->CB16n, list, nl);
  QXD_CHECK_LAUNCH(lat, "k_clover_low");
  k_clover_low<<<grid_cap(2 * nl, 128), 128, 0, lat->stream>>>(g, lat->Ci64, lat->Ci32, lat->Ci16, lat->Ci16n,
                                                               lat->CiB16, lat->CiB16n, list, nl);
  QXD_CHECK_LAUNCH(lat, "k_clover_low");
  return QXD_OK;
}

// Device clover [2][2][18][sv] -> boundary [V][2][36] in the lattice's site order.
__global__ void k_clover_export(Geom g, int order, const double2* __restrict__ C, double2* __restrict__ bnd) {
  i64 n = 2 * g.Vh * 36;  // (site, block, pair)
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    i64 site = t / 36;
    int r = (int)(t - site * 36);
    int blkid = r / 18, k = r - blkid * 18;
    int par;
    i64 cb;
    if (order == QXD_ORDER_IPT) {
      int x[4];
      ipt_coords(g.L, g.B, site, x);
      par = (x[0] + x[1] + x[2] + x[3]) & 1;
      cb = lexi(g, x) >> 1;
    } else {
      i64 u = site;
      int x3 = (int)(u % g.L[3]);
      u /= g.L[3];
      int x2 = (int)(u % g.L[2]);
      u /= g.L[2];
      int x1 = (int)(u % g.L[1]);
      int x0 = (int)(u / g.L[1]);
      par = (x0 + x1 + x2 + x3) & 1;
      cb = site >> 1;
    }
    bnd[t] = C[(i64)((par * 2 + blkid) * 18 + k) * g.sv + cb];
  }
}

qxd_status clover_export(qxd_lattice* lat, double* bnd) {
  i64 n = lat->V * 36;
  k_clover_export<<<grid_cap(n, 256), 256, 0, lat->stream>>>(lat->g, lat->order, lat->C64, (double2*)bnd);
  QXD_CHECK_LAUNCH(lat, "k_clover_export");
  return QXD_OK;
}

// out = C in on parity par (site-local), FP64 single-parity fields [12][sv].
__global__ void k_clover_apply64(Geom g, int par, const double2* __restrict__ C, const double2* __restrict__ in,
                                 double2* __restrict__ out) {
  for (i64 cb = blockIdx.x * (i64)blockDim.x + threadIdx.x; cb < g.Vh; cb += (i64)gridDim.x * blockDim.x) {
#pragma unroll
    for (int blkid = 0; blkid < 2; ++blkid) {
      double r[36];
      const double2* b = C + (i64)((par * 2 + blkid) * 18) * g.sv + cb;
#pragma unroll
      for (int k = 0; k < 18; ++k) {
        double2 v = b[k * g.sv];
        r[2 * k] = v.x;
        r[2 * k + 1] = v.y;
      }
      cd x[6], y[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        double2 v = in[(6 * blkid + k) * g.sv + cb];
        x[k] = mk(v.x, v.y);
      }
      herm6_apply(r, x, y);
#pragma unroll
      for (int k = 0; k < 6; ++k) out[(6 * blkid + k) * g.sv + cb] = make_double2(y[k].re, y[k].im);
    }
  }
}

qxd_status clover_apply64(qxd_lattice* lat, int par, int which, const double2* in, double2* out) {
  k_clover_apply64<<<grid_cap(lat->Vh, 128), 128, 0, lat->stream>>>(lat->g, par, which ? lat->Ci64 : lat->C64,
                                                                    in, out);
  QXD_CHECK_LAUNCH(lat, "k_clover_apply64");
  return QXD_OK;
}

// out = C in on parity par (site-local), FP32 single-parity fields [6][sv] float4.
__global__ void k_clover_apply32(Geom g, int par, const float4* __restrict__ C, const float4* __restrict__ in,
                                 float4* __restrict__ out) {
  for (i64 cb = blockIdx.x * (i64)blockDim.x + threadIdx.x; cb < g.Vh; cb += (i64)gridDim.x * blockDim.x) {
#pragma unroll
    for (int blkid = 0; blkid < 2; ++blkid) {
      float r[36];
      const float4* b = C + (i64)((par * 2 + blkid) * 9) * g.sv + cb;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        float4 v = b[k * g.sv];
        r[4 * k] = v.x;
        r[4 * k + 1] = v.y;
        r[4 * k + 2] = v.z;
        r[4 * k + 3] = v.w;
      }
      cplx<float> x[6], y[6];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float4 v = in[(3 * blkid + k) * g.sv + cb];
        x[2 * k] = mk(v.x, v.y);
        x[2 * k + 1] = mk(v.z, v.w);
      }
      herm6_apply(r, x, y);
#pragma unroll
      for (int k = 0; k < 3; ++k)
        out[(3 * blkid + k) * g.sv + cb] = make_float4(y[2 * k].re, y[2 * k].im, y[2 * k + 1].re, y[2 * k + 1].im);
    }
  }
}

qxd_status clover_apply32(qxd_lattice* lat, int par, int which, const float4* in, float4* out) {
  k_clover_apply32<<<grid_cap(lat->Vh, 128), 128, 0, lat->stream>>>(lat->g, par, which ? lat->Ci32 : lat->C32,
                                                                    in, out);
  QXD_CHECK_LAUNCH(lat, "k_clover_apply32");
  return QXD_OK;
}

}  // namespace qxd
