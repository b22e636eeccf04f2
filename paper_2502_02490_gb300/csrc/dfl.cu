// Inexact deflation on the GPU: the "DFL" of the DFL_SAP_GCR solver the paper's CPU runs use
// (Sec. 5.1; the paper names the method and gives no detail).  The two-level method:
//
//   subspace   Ns fields psi_k (approximate low modes, e.g. random fields improved by SAP
//              inverse iteration, qxd_dfl_generate), restricted to deflation blocks Lambda and
//              orthonormalised block by block (modified Gram-Schmidt in vector order over the
//              12 |Lambda| components): basis psi_{Lambda,k}, P c = sum c_{Lambda,k} psi_{Lambda,k};
//   little D   A = P^+ D P, which couples a block only to itself and its face neighbours:
//              A[(b,k),(b',k')] = <psi_{b,k}, D psi_{b',k'}>, stored per block and neighbour slot;
//   precond    z = P A^-1 P^+ r (inexact coarse solve), then z += M_SAP (r - D z), inside FGCR.
//
// Everything that defines P and A is FP64 (so A can be compared entry by entry with a plain FP64
// construction); the preconditioner applies them to the FP32 fields of the inner solver.
//
// Blocks: extents b_mu dividing L_mu, a block grid n_mu that is 1 or even, b_mu >= 2 where
// n_mu > 1 (the two faces of a block in direction mu must be different site layers), and with C*
// the physical L1 an even number of x blocks and at least two blocks in y and in z.  A block's colour is the 4-bit pattern of its block
// coordinates' parities; a block's face neighbour in direction mu has the colour with bit mu
// flipped, and no other block of that colour touches it.  So for each colour c and vector k', the
// field F = sum over blocks of colour c of psi_{b',k'} gives D F, whose inner products with the
// basis on the self block (c = colour(b)) or on one face layer of b (c = colour(b) ^ (1 << mu))
// are exactly the entries of A.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "dfl.cuh"
#include "reduce.cuh"
#include "trace.cuh"

namespace qxd {

qxd_status apply_D64(qxd_lattice* lat, const double2* in, double2* out);

static void dfl_release(void* p) {
  DflState* d = (DflState*)p;
  void* b[] = {d->basis, d->basis32, d->A, d->nbr, d->cw, d->cpart};
  for (void* q : b)
    if (q) cudaFree(q);
  if (d->hcs) cudaFreeHost(d->hcs);
  delete d;
}

bool dfl_ready(const qxd_lattice* lat) {
  return lat->dfl != nullptr && ((const DflState*)lat->dfl)->epoch == lat->epoch;
}

static qxd_status dfl_geometry(qxd_lattice* lat, const int b[4], DflGeom* dg) {
  const Geom& g = lat->g;
  dg->vb = 1;
  dg->nb = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (b[mu] < 1 || g.L[mu] % b[mu]) return fail(lat, QXD_EINVAL, "deflation block extents must divide the lattice");
    dg->b[mu] = b[mu];
    dg->n[mu] = g.L[mu] / b[mu];
    if (dg->n[mu] != 1 && dg->n[mu] % 2)
      return fail(lat, QXD_EINVAL, "deflation needs a block grid of 1 or an even number of blocks per direction");
    if (dg->n[mu] > 1 && b[mu] < 2)
      return fail(lat, QXD_EINVAL, "deflation blocks need extent >= 2 where the grid has more than one block");
    dg->vb *= b[mu];
    dg->nb *= dg->n[mu];
  }
  if (g.shift && g.shift % (2 * b[1]))
    return fail(lat, QXD_EINVAL, "deflation with C*: the physical L1 must be an even number of x blocks");
  // with C*, a hop across the y or z boundary lands on the x-shifted copy; with a single block in
  // that direction it would reach another block of the same colour, which the colour classes
  // cannot tell apart from the block itself
  if (g.shift && (dg->n[2] < 2 || dg->n[3] < 2))
    return fail(lat, QXD_EINVAL, "deflation with C*: at least two blocks in y and in z");
  if (dg->vb > DFL_MAXVB) return fail(lat, QXD_EINVAL, "deflation block volume must be at most 256 sites");
  dg->stride[3] = 1;
  for (int mu = 2; mu >= 0; --mu) dg->stride[mu] = dg->stride[mu + 1] * b[mu + 1];
  return QXD_OK;
}

// neighbour block of kb in direction mu (dir +-1), with the C* shift of x across the y and z
// boundaries (shift = physical L1 in sites, a whole number of x blocks)
static int block_neighbour(const DflGeom& dg, int shift, const int kb[4], int mu, int dir) {
  int y[4] = {kb[0], kb[1], kb[2], kb[3]};
  y[mu] += dir;
  bool crossed = false;
  if (y[mu] >= dg.n[mu]) {
    y[mu] = 0;
    crossed = true;
  } else if (y[mu] < 0) {
    y[mu] = dg.n[mu] - 1;
    crossed = true;
  }
  if (crossed && shift && mu >= 2) y[1] = (y[1] + shift / dg.b[1]) % dg.n[1];
  return block_index(dg, y);
}

// the thread's site: local index s of block t -> global coordinates, parity and checkerboard index
__device__ __forceinline__ void block_site(const Geom& g, const DflGeom& dg, int t, int s, int lc[4], int& par,
                                           i64& cb) {
  int kb[4];
  block_coords(dg, t, kb);
  int u = s, x[4];
  for (int mu = 3; mu >= 0; --mu) {
    lc[mu] = u % dg.b[mu];
    u /= dg.b[mu];
  }
  for (int mu = 0; mu < 4; ++mu) x[mu] = kb[mu] * dg.b[mu] + lc[mu];
  par = (x[0] + x[1] + x[2] + x[3]) & 1;
  cb = lexi(g, x) >> 1;
}

// Modified Gram-Schmidt of the ns vectors on every block (one CTA per block, one thread per
// block site): w_k -= <u_j, w_k> u_j for j < k in order, then u_k = w_k / ||w_k||.  A vector
// that the projections reduce to rounding (||w_k|| <= 1e-12 of its norm before them) sets *bad.
__global__ void __launch_bounds__(DFL_MAXVB) k_dfl_orthonormalise(Geom g, DflGeom dg, int ns, double2* __restrict__ V,
                                                                  int* __restrict__ bad) {
  __shared__ double sh[2 * 8];
  const int t = blockIdx.x, s = threadIdx.x;
  const bool act = s < dg.vb;  // the CTA is rounded up to whole warps; the extra threads only reduce
  int lc[4], par = 0;
  i64 cb = 0;
  if (act) block_site(g, dg, t, s, lc, par, cb);
  const i64 fs = 24 * g.sv;  // one full field
  const i64 base = (i64)par * 12 * g.sv + cb;
  for (int k = 0; k < ns; ++k) {
    double2* wk = V + (i64)k * fs + base;
    double n0[1] = {0.0};  // ||w_k||^2 before the projections
    if (act)
      for (int c = 0; c < 12; ++c) {
        const double2 b = wk[c * g.sv];
        n0[0] += b.x * b.x + b.y * b.y;
      }
    cta_sum<1>(n0, sh);
    for (int j = 0; j < k; ++j) {
      const double2* uj = V + (i64)j * fs + base;
      double v[2] = {0.0, 0.0};
      if (act)
        for (int c = 0; c < 12; ++c) {
          const double2 a = uj[c * g.sv], b = wk[c * g.sv];
          v[0] += a.x * b.x + a.y * b.y;  // conj(a) b
          v[1] += a.x * b.y - a.y * b.x;
        }
      cta_sum<2>(v, sh);
      if (act)
        for (int c = 0; c < 12; ++c) {
          const double2 a = uj[c * g.sv];
          double2 b = wk[c * g.sv];
          b.x -= v[0] * a.x - v[1] * a.y;
          b.y -= v[0] * a.y + v[1] * a.x;
          wk[c * g.sv] = b;
        }
    }
    double nn[1] = {0.0};
    if (act)
      for (int c = 0; c < 12; ++c) {
        const double2 b = wk[c * g.sv];
        nn[0] += b.x * b.x + b.y * b.y;
      }
    cta_sum<1>(nn, sh);
    // dependent on this block: what the projections leave is rounding (relative 1e-12 or less)
    if (!(nn[0] > 1e-24 * n0[0])) {
      if (s == 0) atomicOr(bad, 1);
      return;  // uniform over the CTA
    }
    const double inv = 1.0 / sqrt(nn[0]);
    if (act)
      for (int c = 0; c < 12; ++c) {
        double2 b = wk[c * g.sv];
        wk[c * g.sv] = make_double2(b.x * inv, b.y * inv);
      }
  }
}

// F = the k'-th subspace field on the blocks of colour c, zero elsewhere (one thread per site)
__global__ void k_dfl_colour_field(Geom g, DflGeom dg, int c, const double2* __restrict__ psi, double2* __restrict__ F) {
  const i64 n = 2 * g.Vh;
  for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < n; e += (i64)gridDim.x * blockDim.x) {
    const int par = e >= g.Vh ? 1 : 0;
    const i64 cb = e - (i64)par * g.Vh;
    int x[4], kb[4];
    cb_coords(g, cb, par, x);
    for (int mu = 0; mu < 4; ++mu) kb[mu] = x[mu] / dg.b[mu];
    const bool on = block_colour(kb) == c;
    const i64 base = (i64)par * 12 * g.sv + cb;
#pragma unroll
    for (int k = 0; k < 12; ++k) F[base + k * g.sv] = on ? psi[base + k * g.sv] : make_double2(0.0, 0.0);
  }
}

// Entries of A from G = D F (F = vector kp on the blocks of colour c): on a block of colour c the
// self slot, <psi_{b,k}, G> over the block; on a block whose colour differs from c in bit mu only,
// the +mu slot over its last layer in mu and the -mu slot over its first layer.
__global__ void __launch_bounds__(DFL_MAXVB) k_dfl_little(Geom g, DflGeom dg, int ns, int c, int kp,
                                                          const double2* __restrict__ V, const double2* __restrict__ G,
                                                          double2* __restrict__ A) {
  __shared__ double sh[4 * 8];
  const int t = blockIdx.x, s = threadIdx.x;
  int kb[4];
  block_coords(dg, t, kb);
  const int d = block_colour(kb) ^ c;
  int mu = -1;
  if (d != 0) {
    if (d & (d - 1)) return;  // more than one bit: no block of colour c touches this one
    mu = d == 1 ? 0 : d == 2 ? 1 : d == 4 ? 2 : 3;
  }
  const bool act = s < dg.vb;
  int lc[4] = {0, 0, 0, 0}, par = 0;
  i64 cb = 0;
  if (act) block_site(g, dg, t, s, lc, par, cb);
  const i64 fs = 24 * g.sv, base = (i64)par * 12 * g.sv + cb;
  // weights of this site in the two sums: the whole block (self), or the +mu / -mu face layers
  const bool in0 = act && (mu < 0 || lc[mu] == dg.b[mu] - 1);
  const bool in1 = act && mu >= 0 && lc[mu] == 0;
  double2 gx[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) gx[q] = act ? G[base + q * g.sv] : make_double2(0.0, 0.0);
  for (int k = 0; k < ns; ++k) {
    const double2* u = V + (i64)k * fs + base;
    double re = 0.0, im = 0.0;
    if (act)
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        const double2 a = u[q * g.sv];
        re += a.x * gx[q].x + a.y * gx[q].y;
        im += a.x * gx[q].y - a.y * gx[q].x;
      }
    double v[4] = {in0 ? re : 0.0, in0 ? im : 0.0, in1 ? re : 0.0, in1 ? im : 0.0};
    cta_sum<4>(v, sh);
    if (s == 0) {
      const int s0 = mu < 0 ? 0 : 1 + 2 * mu;
      A[(((i64)t * DFL_SLOTS + s0) * ns + k) * ns + kp] = make_double2(v[0], v[1]);
      if (mu >= 0) A[(((i64)t * DFL_SLOTS + 2 + 2 * mu) * ns + k) * ns + kp] = make_double2(v[2], v[3]);
    }
  }
}

// ---- coarse vectors (n = nb ns complex, FP64) ----
// y = A x: one thread per (block, k)
__global__ void k_dfl_cmv(int nb, int ns, const double2* __restrict__ A, const int* __restrict__ nbr,
                          const double2* __restrict__ x, double2* __restrict__ y) {
  const i64 n = (i64)nb * ns;
  for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < n; e += (i64)gridDim.x * blockDim.x) {
    const int b = (int)(e / ns), k = (int)(e % ns);
    double re = 0.0, im = 0.0;
    for (int sl = 0; sl < DFL_SLOTS; ++sl) {
      const double2* row = A + (((i64)b * DFL_SLOTS + sl) * ns + k) * ns;
      const double2* xb = x + (i64)nbr[b * DFL_SLOTS + sl] * ns;
      for (int kp = 0; kp < ns; ++kp) {
        const double2 a = row[kp], v = xb[kp];
        re += a.x * v.x - a.y * v.y;
        im += a.x * v.y + a.y * v.x;
      }
    }
    y[e] = make_double2(re, im);
  }
}

// out[j] = <Q_j, v> for j < nq (Q_j at Q + j n), one CTA per j; fixed order
__global__ void __launch_bounds__(256) k_dfl_cdots(const double2* __restrict__ Q, i64 n, int nq,
                                                   const double2* __restrict__ v, double2* __restrict__ out) {
  __shared__ double sh[2 * 8];
  const int j = blockIdx.x;
  const double2* q = Q + (i64)j * n;
  double a[2] = {0.0, 0.0};
  for (i64 i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 x = q[i], y = v[i];
    a[0] += x.x * y.x + x.y * y.y;
    a[1] += x.x * y.y - x.y * y.x;
  }
  cta_sum<2>(a, sh);
  if (threadIdx.x == 0) out[j] = make_double2(a[0], a[1]);
}

// y = a x + y (complex a from device memory, optionally negated)
__global__ void k_dfl_caxpy(i64 n, const double2* __restrict__ a, double sign, const double2* __restrict__ x,
                            double2* __restrict__ y) {
  const double ar = sign * a->x, ai = sign * a->y;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    double2 w = y[i];
    w.x += ar * v.x - ai * v.y;
    w.y += ar * v.y + ai * v.x;
    y[i] = w;
  }
}

// v *= 1 / sqrt(nn->x)  (nn: a <q, q> slot)
__global__ void k_dfl_cscale(i64 n, const double2* __restrict__ nn, double2* __restrict__ v, double2* __restrict__ w) {
  const double s = 1.0 / sqrt(nn->x);
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double2 a = v[i], b = w[i];
    v[i] = make_double2(a.x * s, a.y * s);
    w[i] = make_double2(b.x * s, b.y * s);
  }
}

// ---- fine <-> coarse ----
// The preconditioner applies P and P^+ to the FP32 fields of the inner solver with an FP32 copy
// of the (FP64-orthonormalised) basis, V32 [ns][2][6][sv] float4: FP32 products, FP64 block sums.
// f[b][k] = <psi_{b,k}, r> over block b (r: full FP32 field); one CTA per block, eight basis
// vectors per block reduction
__global__ void __launch_bounds__(DFL_MAXVB) k_dfl_restrict(Geom g, DflGeom dg, int ns, const float4* __restrict__ V,
                                                            const float4* __restrict__ r, double2* __restrict__ f) {
  __shared__ double sh[16 * 8];
  const int t = blockIdx.x, s = threadIdx.x;
  const bool act = s < dg.vb;
  int lc[4], par = 0;
  i64 cb = 0;
  if (act) block_site(g, dg, t, s, lc, par, cb);
  const i64 fs = 12 * g.sv, base = (i64)par * 6 * g.sv + cb;
  float4 rx[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) rx[j] = act ? r[base + j * g.sv] : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k0 = 0; k0 < ns; k0 += 8) {
    double v[16];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      float re = 0.f, im = 0.f;
      if (act && k0 + kk < ns) {
        const float4* u = V + (i64)(k0 + kk) * fs + base;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const float4 a = u[j * g.sv], x = rx[j];
          re += a.x * x.x + a.y * x.y + a.z * x.z + a.w * x.w;  // conj(a) x
          im += a.x * x.y - a.y * x.x + a.z * x.w - a.w * x.z;
        }
      }
      v[2 * kk] = re;
      v[2 * kk + 1] = im;
    }
    cta_sum<16>(v, sh);
    if (s == 0)
      for (int kk = 0; kk < 8 && k0 + kk < ns; ++kk) f[(i64)t * ns + k0 + kk] = make_double2(v[2 * kk], v[2 * kk + 1]);
  }
}

// z = P c (full FP32 field, FP32 basis copy); one thread per site, grid = blocks
__global__ void __launch_bounds__(DFL_MAXVB) k_dfl_prolong(Geom g, DflGeom dg, int ns, const float4* __restrict__ V,
                                                           const double2* __restrict__ c, float4* __restrict__ z) {
  const int t = blockIdx.x, s = threadIdx.x;
  if (s >= dg.vb) return;  // no reduction in this kernel
  int lc[4], par;
  i64 cb;
  block_site(g, dg, t, s, lc, par, cb);
  const i64 fs = 12 * g.sv, base = (i64)par * 6 * g.sv + cb;
  float4 acc[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k = 0; k < ns; ++k) {
    const double2 cd = c[(i64)t * ns + k];
    const float cr = (float)cd.x, ci = (float)cd.y;
    const float4* u = V + (i64)k * fs + base;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float4 a = u[j * g.sv];
      acc[j].x = fmaf(cr, a.x, fmaf(-ci, a.y, acc[j].x));
      acc[j].y = fmaf(cr, a.y, fmaf(ci, a.x, acc[j].y));
      acc[j].z = fmaf(cr, a.z, fmaf(-ci, a.w, acc[j].z));
      acc[j].w = fmaf(cr, a.w, fmaf(ci, a.z, acc[j].w));
    }
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) z[base + j * g.sv] = acc[j];
}

__global__ void k_dfl_scale32(i64 n, const double* __restrict__ nn, float4* __restrict__ v) {
  const float s = (float)(1.0 / sqrt(*nn));
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    float4 a = v[i];
    v[i] = make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
  }
}

#define DTRY(x)                      \
  do {                               \
    qxd_status _s = (x);             \
    if (_s != QXD_OK) return _s;     \
  } while (0)

// Coarse GCR(m) on A c = f in FP64 (classical Gram-Schmidt against normalised A-images, restart
// every m steps), to ||f - A c|| <= coarse_tol ||f|| or coarse_maxiter steps; inexact by design
// (the result only preconditions the outer flexible GCR).
static qxd_status coarse_solve(qxd_lattice* lat, DflState* d, const double2* f, double2* c) {
  const i64 n = (i64)d->dg.nb * d->ns;
  const int m = d->m;
  cudaStream_t S = lat->stream;
  double2* P = d->cw;
  double2* Q = d->cw + (i64)m * n;
  double2* r = d->cw + (i64)2 * m * n;
  double2* dots = (double2*)d->cpart;  // [m] betas, [m] |q|^2, [m + 1] alpha, [m + 2] |r|^2
  QXD_CUDA(lat, cudaMemcpyAsync(r, f, sizeof(double2) * n, cudaMemcpyDeviceToDevice, S));
  QXD_CUDA(lat, cudaMemsetAsync(c, 0, sizeof(double2) * n, S));
  auto rnorm = [&](double* out) -> qxd_status {
    k_dfl_cdots<<<1, 256, 0, S>>>(r, n, 1, r, dots + m + 2);
    QXD_CHECK_LAUNCH(lat, "k_dfl_cdots");
    QXD_CUDA(lat, cudaMemcpyAsync(d->hcs, dots + m + 2, sizeof(double2), cudaMemcpyDeviceToHost, S));
    QXD_CUDA(lat, cudaStreamSynchronize(S));
    *out = std::sqrt(d->hcs[0]);
    return QXD_OK;
  };
  double fn;
  DTRY(rnorm(&fn));
  const double target = d->coarse_tol * fn;
  double rn = fn;
  int it = 0;
  while (rn > target && it < d->coarse_maxiter && std::isfinite(rn)) {
    const int k = it % m;
    double2 *pk = P + (i64)k * n, *qk = Q + (i64)k * n;
    QXD_CUDA(lat, cudaMemcpyAsync(pk, r, sizeof(double2) * n, cudaMemcpyDeviceToDevice, S));
    k_dfl_cmv<<<egrid(n), 256, 0, S>>>(d->dg.nb, d->ns, d->A, d->nbr, pk, qk);
    QXD_CHECK_LAUNCH(lat, "k_dfl_cmv");
    if (k > 0) {
      k_dfl_cdots<<<k, 256, 0, S>>>(Q, n, k, qk, dots);
      QXD_CHECK_LAUNCH(lat, "k_dfl_cdots");
      for (int j = 0; j < k; ++j) {
        k_dfl_caxpy<<<egrid(n), 256, 0, S>>>(n, dots + j, -1.0, Q + (i64)j * n, qk);
        k_dfl_caxpy<<<egrid(n), 256, 0, S>>>(n, dots + j, -1.0, P + (i64)j * n, pk);
      }
      QXD_CHECK_LAUNCH(lat, "k_dfl_caxpy");
    }
    k_dfl_cdots<<<1, 256, 0, S>>>(qk, n, 1, qk, dots + m);
    k_dfl_cscale<<<egrid(n), 256, 0, S>>>(n, dots + m, qk, pk);
    k_dfl_cdots<<<1, 256, 0, S>>>(qk, n, 1, r, dots + m + 1);
    k_dfl_caxpy<<<egrid(n), 256, 0, S>>>(n, dots + m + 1, 1.0, pk, c);
    k_dfl_caxpy<<<egrid(n), 256, 0, S>>>(n, dots + m + 1, -1.0, qk, r);
    QXD_CHECK_LAUNCH(lat, "coarse GCR step");
    DTRY(rnorm(&rn));
    ++it;
  }
  d->coarse_iters += it;
  d->coarse_calls += 1;
  if (!std::isfinite(rn)) return fail(lat, QXD_ENOCONV, "non-finite residual in the coarse solve");
  return QXD_OK;
}

// z = P A^-1 P^+ r, then z += M_SAP (r - D z); full FP32 fields.  Scratch: work slots 58 (D z,
// then the SAP correction) and 59 (r - D z).
qxd_status dfl_precond32(qxd_lattice* lat, const SapSpec& sap, const float4* r, float4* z) {
  DflState* d = (DflState*)lat->dfl;
  if (!d) return fail(lat, QXD_ESTATE, "deflation subspace not set up (qxd_dfl_setup)");
  if (d->epoch != lat->epoch) return fail(lat, QXD_ESTATE, "deflation subspace is stale: the field changed since qxd_dfl_setup");
  const i64 sv = lat->sv, n4 = 12 * sv, n = (i64)d->dg.nb * d->ns;
  const size_t fb = sizeof(float4) * n4;
  float4 *dz, *t;
  DTRY(ensure_work(lat, 58, fb, (void**)&dz));
  DTRY(ensure_work(lat, 59, fb, (void**)&t));
  double2* f = d->cw + (i64)(2 * d->m + 1) * n;
  double2* c = d->cw + (i64)(2 * d->m + 2) * n;
  const int nt = dfl_threads(d->dg);
  k_dfl_restrict<<<d->dg.nb, nt, 0, lat->stream>>>(lat->g, d->dg, d->ns, d->basis32, r, f);
  QXD_CHECK_LAUNCH(lat, "k_dfl_restrict");
  DTRY(coarse_solve(lat, d, f, c));
  k_dfl_prolong<<<d->dg.nb, nt, 0, lat->stream>>>(lat->g, d->dg, d->ns, d->basis32, c, z);
  QXD_CHECK_LAUNCH(lat, "k_dfl_prolong");
  DTRY(hop32(lat, 0, EPI_DFULL, 0, z + 6 * sv, z, dz, 0.f));
  DTRY(hop32(lat, 1, EPI_DFULL, 0, z, z + 6 * sv, dz + 6 * sv, 0.f));
  DTRY(blas_copy(lat, t, r, fb));
  DTRY(blas_axpy_32(lat, -1.0f, dz, t, n4));
  DTRY(sap32(lat, sap.block, sap.ncy, sap.nmr, t, dz));
  return blas_axpy_32(lat, 1.0f, dz, z, n4);
}

}  // namespace qxd

using namespace qxd;

extern "C" {

qxd_status qxd_dfl_setup(qxd_lattice* lat, const int block[4], int ns, const double* vectors, int on_device,
                         double coarse_tol, int coarse_maxiter) {
  QXD_TRACE();
  if (!lat) return QXD_EINVAL;
  if (!block || !vectors) return fail(lat, QXD_EINVAL, "null argument");
  if (ns < 1 || ns > 64) return fail(lat, QXD_EINVAL, "ns must be 1..64");
  if (!(coarse_tol > 0.0) || coarse_maxiter < 1) return fail(lat, QXD_EINVAL, "coarse_tol > 0 and coarse_maxiter >= 1");
  if (!lat->have_clover) return fail(lat, QXD_ESTATE, "dfl_setup before build_clover");
  DflGeom dg;
  DTRY(dfl_geometry(lat, block, &dg));
  if (lat->dfl) {
    lat->dfl_release(lat->dfl);
    lat->dfl = nullptr;
  }
  DflState* d = new DflState();
  d->dg = dg;
  d->ns = ns;
  d->coarse_tol = coarse_tol;
  d->coarse_maxiter = coarse_maxiter;
  const i64 sv = lat->sv, fs = 24 * sv, n = (i64)dg.nb * ns;
  const size_t abytes = sizeof(double2) * (size_t)dg.nb * DFL_SLOTS * ns * ns;
  bool ok = cudaMalloc(&d->basis, sizeof(double2) * fs * ns) == cudaSuccess &&
            cudaMalloc(&d->basis32, sizeof(float4) * 12 * sv * ns) == cudaSuccess &&
            cudaMalloc(&d->A, abytes) == cudaSuccess &&
            cudaMalloc(&d->nbr, sizeof(int) * dg.nb * DFL_SLOTS) == cudaSuccess &&
            cudaMalloc(&d->cw, sizeof(double2) * (size_t)(2 * d->m + 3) * n) == cudaSuccess &&
            cudaMalloc(&d->cpart, sizeof(double2) * (d->m + 4)) == cudaSuccess &&
            cudaMallocHost(&d->hcs, sizeof(double2) * 4) == cudaSuccess;
  if (!ok) {
    dfl_release(d);
    return fail(lat, QXD_ENOMEM, "deflation allocation failed");
  }
  auto bail = [&](qxd_status st) {
    dfl_release(d);
    return st;
  };
  // the subspace vectors in the internal layout
  const size_t vb = sizeof(double) * 24 * lat->V;
  void* bi = nullptr;
  if (!on_device) {
    qxd_status st = ensure_work(lat, 26, vb, &bi);
    if (st) return bail(st);
  }
  for (int k = 0; k < ns; ++k) {
    const double* src = vectors + (i64)k * 24 * lat->V;
    if (!on_device) {
      if (cudaMemcpyAsync(bi, src, vb, cudaMemcpyHostToDevice, lat->stream) != cudaSuccess)
        return bail(fail(lat, QXD_ECUDA, "dfl_setup: copy of the vectors"));
      src = (const double*)bi;
    }
    qxd_status st = pack_spinor64(lat, (const double2*)src, d->basis + (i64)k * fs, 0);
    if (st) return bail(st);
  }
  int* bad;
  {
    qxd_status st = ensure_work(lat, 30, sizeof(int), (void**)&bad);
    if (st) return bail(st);
  }
  cudaMemsetAsync(bad, 0, sizeof(int), lat->stream);
  const int nt = dfl_threads(dg);
  k_dfl_orthonormalise<<<dg.nb, nt, 0, lat->stream>>>(lat->g, dg, ns, d->basis, bad);
  if (cudaGetLastError() != cudaSuccess) return bail(fail(lat, QXD_ECUDA, "k_dfl_orthonormalise launch"));
  int hbad = 0;
  cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, lat->stream);
  if (cudaStreamSynchronize(lat->stream) != cudaSuccess) return bail(fail(lat, QXD_ECUDA, "dfl_setup"));
  if (hbad) return bail(fail(lat, QXD_EINVAL, "deflation vectors are linearly dependent on some block"));
  for (int k = 0; k < ns; ++k) {  // the FP32 copy the preconditioner applies
    qxd_status st = f64_to_f32(lat, d->basis + (i64)k * fs, d->basis32 + (i64)k * 12 * sv, 12 * sv);
    if (st) return bail(st);
  }
  // neighbour table and the colours present
  d->hnbr.assign((size_t)dg.nb * DFL_SLOTS, 0);
  bool present[16] = {false};
  for (int t = 0; t < dg.nb; ++t) {
    int kb[4];
    block_coords(dg, t, kb);
    present[block_colour(kb)] = true;
    d->hnbr[t * DFL_SLOTS] = t;
    for (int mu = 0; mu < 4; ++mu) {
      d->hnbr[t * DFL_SLOTS + 1 + 2 * mu] = block_neighbour(dg, lat->g.shift, kb, mu, +1);
      d->hnbr[t * DFL_SLOTS + 2 + 2 * mu] = block_neighbour(dg, lat->g.shift, kb, mu, -1);
    }
  }
  cudaMemcpyAsync(d->nbr, d->hnbr.data(), sizeof(int) * d->hnbr.size(), cudaMemcpyHostToDevice, lat->stream);
  cudaMemsetAsync(d->A, 0, abytes, lat->stream);
  // A = P^+ D P, colour by colour (FP64 D on the whole lattice; scratch: API slots 24, 25)
  double2 *F, *G;
  {
    qxd_status st = ensure_work(lat, 24, sizeof(double2) * fs, (void**)&F);
    if (!st) st = ensure_work(lat, 25, sizeof(double2) * fs, (void**)&G);
    if (st) return bail(st);
  }
  for (int kp = 0; kp < ns; ++kp)
    for (int c = 0; c < 16; ++c) {
      if (!present[c]) continue;
      k_dfl_colour_field<<<egrid(2 * lat->Vh), 256, 0, lat->stream>>>(lat->g, dg, c, d->basis + (i64)kp * fs, F);
      qxd_status st = apply_D64(lat, F, G);
      if (st) return bail(st);
      k_dfl_little<<<dg.nb, nt, 0, lat->stream>>>(lat->g, dg, ns, c, kp, d->basis, G, d->A);
      if (cudaGetLastError() != cudaSuccess) return bail(fail(lat, QXD_ECUDA, "k_dfl_little launch"));
      lat->launches += 2;
    }
  if (cudaStreamSynchronize(lat->stream) != cudaSuccess) return bail(fail(lat, QXD_ECUDA, "dfl_setup"));
  static std::atomic<i64> generation{0};
  d->gen = ++generation;
  d->epoch = lat->epoch;
  lat->dfl = d;
  lat->dfl_release = dfl_release;
  return QXD_OK;
}

qxd_status qxd_dfl_generate(qxd_lattice* lat, const int sap_block[4], int ncy, int nmr, int ns, int n_it,
                            const double* start, double* out, int on_device) {
  QXD_TRACE();
  if (!lat) return QXD_EINVAL;
  if (!sap_block || !start || !out) return fail(lat, QXD_EINVAL, "null argument");
  if (ns < 1 || n_it < 0 || ncy < 1 || nmr < 1) return fail(lat, QXD_EINVAL, "ns >= 1, n_it >= 0, ncy, nmr >= 1");
  if (!lat->have_clover) return fail(lat, QXD_ESTATE, "dfl_generate before build_clover");
  DTRY(sap_check(lat, sap_block));
  const i64 sv = lat->sv, n4 = 12 * sv;
  const size_t vb = sizeof(double) * 24 * lat->V;
  double2 *f64, *g64;
  float4 *a32, *b32;
  DTRY(ensure_work(lat, 24, sizeof(double2) * 24 * sv, (void**)&f64));
  DTRY(ensure_work(lat, 25, sizeof(double2) * 24 * sv, (void**)&g64));
  DTRY(ensure_work(lat, 43, sizeof(float4) * n4, (void**)&a32));
  DTRY(ensure_work(lat, 44, sizeof(float4) * n4, (void**)&b32));
  void *bi = nullptr, *bo = nullptr;
  if (!on_device) {
    DTRY(ensure_work(lat, 26, vb, &bi));
    DTRY(ensure_work(lat, 27, vb, &bo));
  }
  for (int k = 0; k < ns; ++k) {
    const double* src = start + (i64)k * 24 * lat->V;
    double* dst = out + (i64)k * 24 * lat->V;
    if (!on_device) {
      QXD_CUDA(lat, cudaMemcpyAsync(bi, src, vb, cudaMemcpyHostToDevice, lat->stream));
      src = (const double*)bi;
    }
    DTRY(pack_spinor64(lat, (const double2*)src, f64, 0));
    DTRY(f64_to_f32(lat, f64, a32, n4));
    DTRY(blas_norm2_32(lat, a32, n4, SC_TMP0));
    k_dfl_scale32<<<egrid(n4), 256, 0, lat->stream>>>(n4, lat->scal + SC_TMP0, a32);
    QXD_CHECK_LAUNCH(lat, "k_dfl_scale32");
    for (int it = 0; it < n_it; ++it) {  // v <- M_SAP v / ||M_SAP v||
      DTRY(sap32(lat, sap_block, ncy, nmr, a32, b32));
      DTRY(blas_norm2_32(lat, b32, n4, SC_TMP0));
      k_dfl_scale32<<<egrid(n4), 256, 0, lat->stream>>>(n4, lat->scal + SC_TMP0, b32);
      QXD_CHECK_LAUNCH(lat, "k_dfl_scale32");
      std::swap(a32, b32);
    }
    DTRY(f32_to_f64(lat, a32, g64, n4));
    DTRY(unpack_spinor64(lat, g64, on_device ? (double2*)dst : (double2*)bo, 0));
    if (!on_device) {
      QXD_CUDA(lat, cudaMemcpyAsync(dst, bo, vb, cudaMemcpyDeviceToHost, lat->stream));
      QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
    }
  }
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  return QXD_OK;
}

qxd_status qxd_dfl_get_little(qxd_lattice* lat, double* A, int* nbr) {
  QXD_TRACE();
  if (!lat) return QXD_EINVAL;
  DflState* d = (DflState*)lat->dfl;
  if (!d) return fail(lat, QXD_ESTATE, "deflation subspace not set up");
  if (!A || !nbr) return fail(lat, QXD_EINVAL, "null argument");
  const size_t abytes = sizeof(double2) * (size_t)d->dg.nb * DFL_SLOTS * d->ns * d->ns;
  QXD_CUDA(lat, cudaMemcpyAsync(A, d->A, abytes, cudaMemcpyDeviceToHost, lat->stream));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  std::memcpy(nbr, d->hnbr.data(), sizeof(int) * d->hnbr.size());
  return QXD_OK;
}

qxd_status qxd_dfl_info(qxd_lattice* lat, int* nblocks, int* ns, int64_t* coarse_iters, int64_t* coarse_calls) {
  if (!lat) return QXD_EINVAL;
  DflState* d = (DflState*)lat->dfl;
  if (!d) return fail(lat, QXD_ESTATE, "deflation subspace not set up");
  if (nblocks) *nblocks = d->dg.nb;
  if (ns) *ns = d->ns;
  if (coarse_iters) *coarse_iters = d->coarse_iters;
  if (coarse_calls) *coarse_calls = d->coarse_calls;
  return QXD_OK;
}

}  // extern "C"
