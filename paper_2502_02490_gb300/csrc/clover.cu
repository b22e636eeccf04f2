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
#include "qxd_internal.cuh"

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

__device__ __forceinline__ M3 load_u(const Geom& g, const double2* __restrict__ U, const int y[4], int mu) {
  i64 lam = lexi(g, y);
  int par = (y[0] + y[1] + y[2] + y[3]) & 1;
  const double2* b = U + (i64)((par * 4 + mu) * 9) * g.sv + (lam >> 1);
  M3 r;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double2 v = b[k * g.sv];
    r.m[k] = mk(v.x, v.y);
  }
  return r;
}

__device__ __forceinline__ double load_a(const Geom& g, const double* __restrict__ A, const int y[4], int mu) {
  i64 lam = lexi(g, y);
  int par = (y[0] + y[1] + y[2] + y[3]) & 1;
  return A[(i64)(par * 4 + mu) * g.sv + (lam >> 1)];
}

// c = a b, with optional daggers on a and/or b
template <bool DA, bool DB>
__device__ __forceinline__ M3 mul(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cd s = mk(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        cd x = DA ? mk(a.m[3 * k + i].re, -a.m[3 * k + i].im) : a.m[3 * i + k];
        cd y = DB ? mk(b.m[3 * j + k].re, -b.m[3 * j + k].im) : b.m[3 * k + j];
        s = s + cmul(x, y);
      }
      c.m[3 * i + j] = s;
    }
  return c;
}

// Traceless anti-Hermitian Fhat_{mu nu}(x) = (Q - Q^dag)/8 - tr/3 and the U(1) fhat (imaginary part).
__device__ void field_strength(const Geom& g, const double2* __restrict__ U, const double* __restrict__ A,
                               const int x[4], int mu, int nu, M3& F, double& f1) {
  int xp[4], t[4];
  M3 Q;
  double s1 = 0.0;
  // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
  {
    M3 a = load_u(g, U, x, mu);
    for (int i = 0; i < 4; ++i) xp[i] = x[i];
    step(g, xp, mu, +1);
    M3 b = load_u(g, U, xp, nu);
    for (int i = 0; i < 4; ++i) t[i] = x[i];
    step(g, t, nu, +1);
    M3 c = load_u(g, U, t, mu);
    M3 d = load_u(g, U, x, nu);
    Q = mul<false, true>(mul<false, true>(mul<false, false>(a, b), c), d);
    s1 += sin(load_a(g, A, x, mu) + load_a(g, A, xp, nu) - load_a(g, A, t, mu) - load_a(g, A, x, nu));
  }
  // leaf 2: U_nu(x) U_mu(x+nu-mu)^+ U_nu(x-mu)^+ U_mu(x-mu)
  {
    int xm[4], xnm[4];
    for (int i = 0; i < 4; ++i) xm[i] = x[i];
    step(g, xm, mu, -1);
    for (int i = 0; i < 4; ++i) xnm[i] = xm[i];
    step(g, xnm, nu, +1);
    M3 a = load_u(g, U, x, nu);
    M3 b = load_u(g, U, xnm, mu);
    M3 c = load_u(g, U, xm, nu);
    M3 d = load_u(g, U, xm, mu);
    M3 r = mul<false, false>(mul<false, true>(mul<false, true>(a, b), c), d);
#pragma unroll
    for (int k = 0; k < 9; ++k) Q.m[k] = Q.m[k] + r.m[k];
    s1 += sin(load_a(g, A, x, nu) - load_a(g, A, xnm, mu) - load_a(g, A, xm, nu) + load_a(g, A, xm, mu));
  }
  // leaf 3: U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
  {
    int xm[4], xmn[4], xn[4];
    for (int i = 0; i < 4; ++i) xm[i] = x[i];
    step(g, xm, mu, -1);
    for (int i = 0; i < 4; ++i) xmn[i] = xm[i];
    step(g, xmn, nu, -1);
    for (int i = 0; i < 4; ++i) xn[i] = x[i];
    step(g, xn, nu, -1);
    M3 a = load_u(g, U, xm, mu);
    M3 b = load_u(g, U, xmn, nu);
    M3 c = load_u(g, U, xmn, mu);
    M3 d = load_u(g, U, xn, nu);
    M3 ab = mul<true, true>(a, b);
    M3 r = mul<false, false>(mul<false, false>(ab, c), d);
#pragma unroll
    for (int k = 0; k < 9; ++k) Q.m[k] = Q.m[k] + r.m[k];
    s1 += sin(-load_a(g, A, xm, mu) - load_a(g, A, xmn, nu) + load_a(g, A, xmn, mu) + load_a(g, A, xn, nu));
  }
  // leaf 4: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
  {
    int xn[4], xnp[4];
    for (int i = 0; i < 4; ++i) xn[i] = x[i];
    step(g, xn, nu, -1);
    for (int i = 0; i < 4; ++i) xnp[i] = xn[i];
    step(g, xnp, mu, +1);
    M3 a = load_u(g, U, xn, nu);
    M3 b = load_u(g, U, xn, mu);
    M3 c = load_u(g, U, xnp, nu);
    M3 d = load_u(g, U, x, mu);
    M3 r = mul<false, true>(mul<false, false>(mul<true, false>(a, b), c), d);
#pragma unroll
    for (int k = 0; k < 9; ++k) Q.m[k] = Q.m[k] + r.m[k];
    s1 += sin(-load_a(g, A, xn, nu) + load_a(g, A, xn, mu) + load_a(g, A, xnp, nu) - load_a(g, A, x, mu));
  }
  // F = (Q - Q^+)/8, then remove the trace
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cd a = Q.m[3 * i + j], b = Q.m[3 * j + i];
      F.m[3 * i + j] = mk((a.re - b.re) * 0.125, (a.im + b.im) * 0.125);
    }
  double tr_im = (F.m[0].im + F.m[4].im + F.m[8].im) / 3.0;  // trace of an anti-Hermitian matrix is imaginary
  F.m[0].im -= tr_im;
  F.m[4].im -= tr_im;
  F.m[8].im -= tr_im;
  f1 = 0.25 * s1;  // fhat = i f1
}

// blk (6x6, full storage) += s * sigma_l (x) Y,  s complex
__device__ __forceinline__ void add_sigma(cd blk[36], int l, cd s, const cd Y[9]) {
  // sigma_1: (0,1) = 1, (1,0) = 1; sigma_2: (0,1) = -i, (1,0) = i; sigma_3: (0,0) = 1, (1,1) = -1
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cd y = cmul(s, Y[3 * a + b]);
      if (l == 1) {
        blk[(a) * 6 + (3 + b)] = blk[(a) * 6 + (3 + b)] + y;
        blk[(3 + a) * 6 + b] = blk[(3 + a) * 6 + b] + y;
      } else if (l == 2) {
        blk[(a) * 6 + (3 + b)] = blk[(a) * 6 + (3 + b)] + mk(y.im, -y.re);  // -i y
        blk[(3 + a) * 6 + b] = blk[(3 + a) * 6 + b] + timesI(y);
      } else {
        blk[(a) * 6 + b] = blk[(a) * 6 + b] + y;
        blk[(3 + a) * 6 + (3 + b)] = blk[(3 + a) * 6 + (3 + b)] - y;
      }
    }
}

__device__ __forceinline__ void pack_block(const cd blk[36], double r[36]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) r[i] = blk[7 * i].re;
  int k = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      // symmetrise the rounding of the two triangles
      r[6 + 2 * k] = 0.5 * (blk[6 * i + j].re + blk[6 * j + i].re);
      r[7 + 2 * k] = 0.5 * (blk[6 * i + j].im - blk[6 * j + i].im);
      ++k;
    }
}

__global__ void __launch_bounds__(128) k_clover_build(Geom g, const double2* __restrict__ U,
                                                      const double* __restrict__ A, double diag, double csw,
                                                      double cq, double2* __restrict__ C) {
  i64 n = 2 * g.Vh;
  for (i64 s = blockIdx.x * (i64)blockDim.x + threadIdx.x; s < n; s += (i64)gridDim.x * blockDim.x) {
    int par = s >= g.Vh ? 1 : 0;
    i64 cb = s - (i64)par * g.Vh;
    int x[4];
    cb_coords(g, cb, par, x);
    cd Gp[3][9], Gm[3][9];
    double gp[3], gm[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      gp[l] = gm[l] = 0.0;
#pragma unroll
      for (int k = 0; k < 9; ++k) Gp[l][k] = Gm[l][k] = mk(0.0, 0.0);
    }
    // planes: (0,1) (0,2) (0,3) electric; (2,3) -> l=1 (+), (1,3) -> l=2 (-), (1,2) -> l=3 (+)
    for (int p = 0; p < 6; ++p) {
      int mu, nu, l;
      double sgn;
      bool electric;
      if (p < 3) {
        mu = 0; nu = p + 1; l = p; sgn = 1.0; electric = true;
      } else if (p == 3) {
        mu = 2; nu = 3; l = 0; sgn = 1.0; electric = false;
      } else if (p == 4) {
        mu = 1; nu = 3; l = 1; sgn = -1.0; electric = false;
      } else {
        mu = 1; nu = 2; l = 2; sgn = 1.0; electric = false;
      }
      M3 F;
      double f1;
      field_strength(g, U, A, x, mu, nu, F, f1);
      // G^+ = F_0l - Ftilde_l, G^- = F_0l + Ftilde_l
      double sp = electric ? 1.0 : -sgn, sm = electric ? 1.0 : sgn;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        Gp[l][k] = Gp[l][k] + sp * F.m[k];
        Gm[l][k] = Gm[l][k] + sm * F.m[k];
      }
      gp[l] += sp * f1;
      gm[l] += sm * f1;
    }
    for (int blkid = 0; blkid < 2; ++blkid) {
      cd blk[36];
#pragma unroll
      for (int k = 0; k < 36; ++k) blk[k] = mk(0.0, 0.0);
#pragma unroll
      for (int i = 0; i < 6; ++i) blk[7 * i] = mk(diag, 0.0);
      double side = blkid == 0 ? 0.5 : -0.5;  // +(i/2) on A_+, -(i/2) on A_-
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        cd Y[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          // Y = c_sw G_l + q c_sw^QED g_l 1, where g_l = i * (gp or gm) (fhat is imaginary)
          cd Gv = blkid == 0 ? Gp[l][k] : Gm[l][k];
          Y[k] = csw * Gv;
        }
        double gv = blkid == 0 ? gp[l] : gm[l];
        Y[0].im += cq * gv;
        Y[4].im += cq * gv;
        Y[8].im += cq * gv;
        add_sigma(blk, l + 1, mk(0.0, side), Y);
      }
      double r[36];
      pack_block(blk, r);
      double2* out = C + (i64)((par * 2 + blkid) * 18) * g.sv + cb;
#pragma unroll
      for (int k = 0; k < 18; ++k) out[k * g.sv] = make_double2(r[2 * k], r[2 * k + 1]);
    }
  }
}

// Inverse of each Hermitian 6x6 block by Gauss-Jordan elimination with partial pivoting (FP64).
// A block whose pivot falls below 1e-14 times its largest entry sets *bad (odd sites only).
__global__ void __launch_bounds__(128) k_clover_invert(Geom g, const double2* __restrict__ C,
                                                       double2* __restrict__ Ci, int* __restrict__ bad) {
  i64 n = 2 * g.Vh * 2;
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    int blkid = (int)(t & 1);
    i64 s = t >> 1;
    int par = s >= g.Vh ? 1 : 0;
    i64 cb = s - (i64)par * g.Vh;
    const double2* in = C + (i64)((par * 2 + blkid) * 18) * g.sv + cb;
    double r[36];
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      double2 v = in[k * g.sv];
      r[2 * k] = v.x;
      r[2 * k + 1] = v.y;
    }
    cd a[6][6], inv[6][6];
    double amax = 0.0;
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) inv[i][j] = mk(i == j ? 1.0 : 0.0, 0.0);
    for (int i = 0; i < 6; ++i) {
      a[i][i] = mk(r[i], 0.0);
      amax = fmax(amax, fabs(r[i]));
    }
    int k = 0;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j) {
        a[i][j] = mk(r[6 + 2 * k], r[7 + 2 * k]);
        a[j][i] = mk(r[6 + 2 * k], -r[7 + 2 * k]);
        amax = fmax(amax, fabs(r[6 + 2 * k]) + fabs(r[7 + 2 * k]));
        ++k;
      }
    bool singular = false;
    for (int c = 0; c < 6; ++c) {
      int piv = c;
      double best = -1.0;
      for (int i = c; i < 6; ++i) {
        double m = a[i][c].re * a[i][c].re + a[i][c].im * a[i][c].im;
        if (m > best) {
          best = m;
          piv = i;
        }
      }
      if (!(sqrt(best) > 1e-14 * amax)) singular = true;  // strict: an all-zero block is singular
      if (piv != c) {
        for (int j = 0; j < 6; ++j) {
          cd tmp = a[c][j];
          a[c][j] = a[piv][j];
          a[piv][j] = tmp;
          tmp = inv[c][j];
          inv[c][j] = inv[piv][j];
          inv[piv][j] = tmp;
        }
      }
      cd p = a[c][c];
      double pm = p.re * p.re + p.im * p.im;
      cd pinv = pm > 0.0 ? mk(p.re / pm, -p.im / pm) : mk(0.0, 0.0);
      for (int j = 0; j < 6; ++j) {
        a[c][j] = cmul(a[c][j], pinv);
        inv[c][j] = cmul(inv[c][j], pinv);
      }
      for (int i = 0; i < 6; ++i) {
        if (i == c) continue;
        cd f = a[i][c];
        for (int j = 0; j < 6; ++j) {
          a[i][j] = a[i][j] - cmul(f, a[c][j]);
          inv[i][j] = inv[i][j] - cmul(f, inv[c][j]);
        }
      }
    }
    if (singular && par == 1) atomicOr(bad, 1);
    double o[36];
    for (int i = 0; i < 6; ++i) o[i] = inv[i][i].re;
    k = 0;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j) {
        o[6 + 2 * k] = 0.5 * (inv[i][j].re + inv[j][i].re);
        o[7 + 2 * k] = 0.5 * (inv[i][j].im - inv[j][i].im);
        ++k;
      }
    double2* out = Ci + (i64)((par * 2 + blkid) * 18) * g.sv + cb;
    for (int k2 = 0; k2 < 18; ++k2) out[k2 * g.sv] = make_double2(o[2 * k2], o[2 * k2 + 1]);
  }
}

// FP64 clover [2][2][18][sv] -> FP32 [2][2][9][sv] float4 and 16-bit with one scale per block.
__global__ void k_clover_low(Geom g, const double2* __restrict__ C, float4* __restrict__ C32,
                             uint2* __restrict__ C16, float* __restrict__ C16n, uint2* __restrict__ CB,
                             float* __restrict__ CBn) {
  i64 n = 4 * g.sv;  // (parity, block, site incl. padding)
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    i64 pb = t / g.sv, cb = t - pb * g.sv;
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
  k_clover_build<<<grid_cap(2 * g.Vh, 128), 128, 0, lat->stream>>>(g, lat->U, lat->A, 4.0 + lat->m0, lat->csw,
                                                                   lat->q * lat->csw_qed, lat->C64);
  QXD_CHECK_LAUNCH(lat, "k_clover_build");
  void* w;
  qxd_status st = ensure_work(lat, 30, sizeof(int), &w);  // slot 30: clover singular flag
  if (st) return st;
  int* bad = (int*)w;
  QXD_CUDA(lat, cudaMemsetAsync(bad, 0, sizeof(int), lat->stream));
  k_clover_invert<<<grid_cap(4 * g.Vh, 128), 128, 0, lat->stream>>>(g, lat->C64, lat->Ci64, bad);
  QXD_CHECK_LAUNCH(lat, "k_clover_invert");
  k_clover_low<<<grid_cap(4 * g.sv, 128), 128, 0, lat->stream>>>(g, lat->C64, lat->C32, lat->C16, lat->C16n,
                                                                 lat->CB16, lat->CB16n);
  QXD_CHECK_LAUNCH(lat, "k_clover_low");
  k_clover_low<<<grid_cap(4 * g.sv, 128), 128, 0, lat->stream>>>(g, lat->Ci64, lat->Ci32, lat->Ci16, lat->Ci16n,
                                                                 lat->CiB16, lat->CiB16n);
  QXD_CHECK_LAUNCH(lat, "k_clover_low");
  int hbad = 0;
  QXD_CUDA(lat, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, lat->stream));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  if (hbad) return fail(lat, QXD_ESINGULAR, "a clover block on an odd site is not invertible");
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
      par = site >= g.Vh ? 1 : 0;
      cb = site - (i64)par * g.Vh;
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
