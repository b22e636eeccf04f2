// Three-level multigrid on the GPU: the multigrid GCR of the paper's GPU solves (Sec. 5.1; the
// paper names the method and gives no detail).  Level 1 is the deflation subspace of
// qxd_dfl_setup (csrc/dfl.cu): A1 = P1^+ D P1 on blocks of the fine lattice.  Level 2 aggregates
// a_0 x a_1 x a_2 x a_3 level-1 blocks:
//
//   basis      ns2 level-1 vectors restricted to every aggregate and orthonormalised there
//              (modified Gram-Schmidt in vector order): P2, stored per aggregate [nb2][ns2][E],
//              E = (blocks per aggregate) x ns1 entries in level-1 order within the aggregate;
//   A2         the Galerkin product P2^+ A1 P2, a nearest-neighbour stencil on the aggregate grid
//              [nb2][9][ns2][ns2], formed directly from the stencil of A1: the coupling of block b
//              to b' = b +- mu lands in the self slot of b's aggregate when b' lies in it, else in
//              its +-mu slot;
//   S1         nu minimal-residual steps on A1 from zero (level-1 smoother);
//   G2         n2 GCR steps on A2 from zero (coarsest solve);
//   T1         y = S1 f; y += P2 G2(P2^+ (f - A1 y)); y += S1 (f - A1 y)   (two-grid cycle);
//   K1         n1 flexible GCR steps on A1 from zero, preconditioned by T1 (a K-cycle);
//   fine       z = M_SAP^pre r (ncy_pre cycles, none for 0); z += P1 K1(P1^+ (r - D z));
//              z += M_SAP (r - D z), inside the fine flexible GCR (QXD_SOLVER_MP_MG_GCR).
//
// Both coarse levels are FP64 with every coefficient on the device and fixed step counts, so the
// preconditioner makes no host round trip and the level-1 solve (some 400 small launches) is
// captured once as a CUDA graph and replayed; inner products sum fixed chunks in a fixed order.
// The fine smoothing works on the FP32 fields of the inner solver.  GCR steps: z = M r, w = A z, classical Gram-Schmidt of w against the cycle's
// earlier normalised w_j (the same combination applied to z), w and z divided by ||w||,
// alpha = <w, r>, x += alpha z, r -= alpha w; a step whose w vanishes changes nothing.
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <vector>

#include "dfl.cuh"
#include "trace.cuh"

namespace qxd {

constexpr int MG_MAXNS2 = 32;
constexpr int MG_MAXM = 16;
constexpr int MG_THREADS = 256;
constexpr int MG_DOT_BLOCKS = 64;    // partial sums per inner product (fixed: results do not depend on the GPU)
constexpr int MG_DOT_CHUNK = 2048;   // entries per partial at least

struct MgState {
  int agg[4], n2g[4];
  int nb1, ns1, nb2, ns2, va, E;
  i64 n1, n2;
  double2* P2 = nullptr;    // [nb2][ns2][E]
  double2* A2 = nullptr;    // [nb2][9][ns2][ns2]
  int* nbr2 = nullptr;      // [nb2][9]
  int* agg_of = nullptr;    // [nb1] aggregate of a level-1 block
  int* loc_of = nullptr;    // [nb1] its index within the aggregate (lexicographic, direction 3 fastest)
  int* blk_of = nullptr;    // [nb2][va] level-1 block at a local index
  std::vector<int> hnbr2;
  int nu = 2, n1s = 4, n2s = 8, m = 8, ncy_pre = 0;
  double2* w1 = nullptr;    // level-1 work: K1 Z[m], W[m], r; T1 rho, q, t; f1, c1
  double2* w2 = nullptr;    // level-2 work: G2 Z[m], W[m], r; f2, c2
  double2* sc = nullptr;    // device scalars: K1 [m + 2], G2 [m + 2], MR [2]
  double2* part = nullptr;  // inner-product partials [MG_MAXM][MG_DOT_BLOCKS]
  i64 dfl_gen = -1;         // the deflation set-up it was built on
  i64 coarse_calls = 0;
  // the level-1 solve f1 -> c1 captured once as a CUDA graph (on a private stream: capture is
  // refused on the legacy default stream) and replayed on the lattice stream
  cudaStream_t side = nullptr;
  cudaGraphExec_t k1_exec = nullptr;
  i64 k1_launches = 0;
};

static void mg_release(void* p) {
  MgState* s = (MgState*)p;
  void* b[] = {s->P2, s->A2, s->nbr2, s->agg_of, s->loc_of, s->blk_of, s->w1, s->w2, s->sc, s->part};
  for (void* q : b)
    if (q) cudaFree(q);
  if (s->k1_exec) cudaGraphExecDestroy(s->k1_exec);
  if (s->side) cudaStreamDestroy(s->side);
  delete s;
}

bool mg_ready(const qxd_lattice* lat) {
  if (!lat->mg || !dfl_ready(lat)) return false;
  return ((const MgState*)lat->mg)->dfl_gen == ((const DflState*)lat->dfl)->gen;
}

// ---- coarse-vector kernels (n complex entries, FP64) ----

// y = A x (f == nullptr) or y = f - A x: one thread per (block, k) of a stencil operator
__global__ void k_mg_cmv(int nb, int ns, const double2* __restrict__ A, const int* __restrict__ nbr,
                         const double2* __restrict__ x, const double2* __restrict__ f, double2* __restrict__ y) {
  const i64 n = (i64)nb * ns;
  for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < n; e += (i64)gridDim.x * blockDim.x) {
    const int b = (int)(e / ns), k = (int)(e % ns);
    double re = 0.0, im = 0.0;
    for (int sl = 0; sl < DFL_SLOTS; ++sl) {
      const double2* row = A + (((i64)b * DFL_SLOTS + sl) * ns + k) * ns;
      const double2* xb = x + (i64)nbr[b * DFL_SLOTS + sl] * ns;
      for (int kp = 0; kp < ns; ++kp) {
        const double2 a = row[kp], v = xb[kp];
        re = fma(a.x, v.x, re);
        re = fma(-a.y, v.y, re);
        im = fma(a.x, v.y, im);
        im = fma(a.y, v.x, im);
      }
    }
    y[e] = f ? make_double2(f[e].x - re, f[e].y - im) : make_double2(re, im);
  }
}

// partial inner products <Q_j, v> (Q_j at Q + j n) over fixed chunks: block (b, j) sums entries
// b chunk .. (b + 1) chunk - 1 in a fixed order into part[j][b]
__global__ void __launch_bounds__(256) k_mg_dots_part(const double2* __restrict__ Q, i64 n, i64 chunk,
                                                      const double2* __restrict__ v, double2* __restrict__ part) {
  __shared__ double sh[2 * 8];
  const int b = blockIdx.x, j = blockIdx.y;
  const double2* q = Q + (i64)j * n;
  const i64 lo = (i64)b * chunk, hi = lo + chunk < n ? lo + chunk : n;
  double a[2] = {0.0, 0.0};
  for (i64 i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double2 x = q[i], y = v[i];
    a[0] += x.x * y.x + x.y * y.y;
    a[1] += x.x * y.y - x.y * y.x;
  }
  cta_sum<2>(a, sh);
  if (threadIdx.x == 0) part[(i64)j * MG_DOT_BLOCKS + b] = make_double2(a[0], a[1]);
}

// out[j] = sum of the nb partials of product j, in block order (one warp per product)
__global__ void k_mg_dots_fin(const double2* __restrict__ part, int nb, double2* __restrict__ out) {
  const int j = blockIdx.x, lane = threadIdx.x;
  double re = lane < nb ? part[(i64)j * MG_DOT_BLOCKS + lane].x : 0.0;
  double im = lane < nb ? part[(i64)j * MG_DOT_BLOCKS + lane].y : 0.0;
  if (lane + 32 < nb) {
    re += part[(i64)j * MG_DOT_BLOCKS + lane + 32].x;
    im += part[(i64)j * MG_DOT_BLOCKS + lane + 32].y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) out[j] = make_double2(re, im);
}

// w -= sum_j c_j W_j and z -= sum_j c_j Z_j for j < k (c: k device slots)
__global__ void k_mg_orth(i64 n, int k, const double2* __restrict__ c, const double2* __restrict__ W,
                          const double2* __restrict__ Z, double2* __restrict__ w, double2* __restrict__ z) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double2 a = w[i], b = z[i];
    for (int j = 0; j < k; ++j) {
      const double2 cj = c[j], u = W[(i64)j * n + i], v = Z[(i64)j * n + i];
      a.x -= cj.x * u.x - cj.y * u.y;
      a.y -= cj.x * u.y + cj.y * u.x;
      b.x -= cj.x * v.x - cj.y * v.y;
      b.y -= cj.x * v.y + cj.y * v.x;
    }
    w[i] = a;
    z[i] = b;
  }
}

// w, z *= 1 / sqrt(nn) (nn: a <w, w> slot; 0 when it vanishes)
__global__ void k_mg_scale(i64 n, const double2* __restrict__ nn, double2* __restrict__ w, double2* __restrict__ z) {
  const double s = nn->x > 0.0 ? 1.0 / sqrt(nn->x) : 0.0;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    const double2 a = w[i], b = z[i];
    w[i] = make_double2(a.x * s, a.y * s);
    z[i] = make_double2(b.x * s, b.y * s);
  }
}

// v *= 1 / sqrt(nn) (nn: a <v, v> slot; 0 when it vanishes)
__global__ void k_mg_scale1(i64 n, const double2* __restrict__ nn, double2* __restrict__ v) {
  const double s = nn->x > 0.0 ? 1.0 / sqrt(nn->x) : 0.0;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    const double2 a = v[i];
    v[i] = make_double2(a.x * s, a.y * s);
  }
}

// x += alpha z, r -= alpha w (alpha: a device slot)
__global__ void k_mg_axpy2(i64 n, const double2* __restrict__ al, const double2* __restrict__ z, double2* __restrict__ x,
                           const double2* __restrict__ w, double2* __restrict__ r) {
  const double ar = al->x, ai = al->y;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    const double2 u = z[i], v = w[i];
    double2 a = x[i], b = r[i];
    a.x += ar * u.x - ai * u.y;
    a.y += ar * u.y + ai * u.x;
    b.x -= ar * v.x - ai * v.y;
    b.y -= ar * v.y + ai * v.x;
    x[i] = a;
    r[i] = b;
  }
}

// one MR step: alpha = <q, rho> / <q, q> (d[0], d[1]; 0 when q vanishes); y += alpha rho, rho -= alpha q
__global__ void k_mg_mr(i64 n, const double2* __restrict__ d, double2* __restrict__ rho, const double2* __restrict__ q,
                        double2* __restrict__ y) {
  const double qq = d[1].x;
  const double ar = qq > 0.0 ? d[0].x / qq : 0.0, ai = qq > 0.0 ? d[0].y / qq : 0.0;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    const double2 u = rho[i], v = q[i];
    double2 a = y[i];
    a.x += ar * u.x - ai * u.y;
    a.y += ar * u.y + ai * u.x;
    y[i] = a;
    rho[i] = make_double2(u.x - (ar * v.x - ai * v.y), u.y - (ar * v.y + ai * v.x));
  }
}

// f2[g][k2] = sum over the aggregate's entries of conj(P2[g][k2][e]) f1[entry e]; one thread per (g, k2)
__global__ void k_mg_restrict2(int nb2, int ns2, int E, int ns1, int va, const double2* __restrict__ P2,
                               const int* __restrict__ blk_of, const double2* __restrict__ f1, double2* __restrict__ f2) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nb2 * ns2) return;
  const int g = o / ns2;
  const double2* p = P2 + (i64)o * E;
  double re = 0.0, im = 0.0;
  for (int bl = 0; bl < va; ++bl) {
    const double2* fb = f1 + (i64)blk_of[g * va + bl] * ns1;
    for (int i = 0; i < ns1; ++i) {
      const double2 a = p[bl * ns1 + i], b = fb[i];
      re += a.x * b.x + a.y * b.y;  // conj(a) b
      im += a.x * b.y - a.y * b.x;
    }
  }
  f2[o] = make_double2(re, im);
}

// y1[b][i] += sum_k2 P2[g(b)][k2][loc(b) ns1 + i] c2[g(b)][k2]; one thread per level-1 entry
__global__ void k_mg_prolong2(int nb1, int ns1, int ns2, int E, const double2* __restrict__ P2,
                              const int* __restrict__ agg_of, const int* __restrict__ loc_of,
                              const double2* __restrict__ c2, double2* __restrict__ y1) {
  const i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x;
  if (e >= (i64)nb1 * ns1) return;
  const int b = (int)(e / ns1), i = (int)(e % ns1);
  const int g = agg_of[b], off = loc_of[b] * ns1 + i;
  double2 a = y1[e];
  for (int k = 0; k < ns2; ++k) {
    const double2 p = P2[((i64)g * ns2 + k) * E + off], c = c2[(i64)g * ns2 + k];
    a.x += p.x * c.x - p.y * c.y;
    a.y += p.x * c.y + p.y * c.x;
  }
  y1[e] = a;
}

// P2[g][k][e] = V[k][entry e of aggregate g] (the caller's level-1 vectors)
__global__ void k_mg_gather2(int nb2, int ns2, int E, int ns1, int va, const int* __restrict__ blk_of, i64 n1,
                             const double2* __restrict__ V, double2* __restrict__ P2) {
  const i64 o = blockIdx.x * (i64)blockDim.x + threadIdx.x;
  if (o >= (i64)nb2 * ns2 * E) return;
  const int e = (int)(o % E), k = (int)((o / E) % ns2), g = (int)(o / ((i64)E * ns2));
  const int bl = e / ns1, i = e % ns1;
  P2[o] = V[(i64)k * n1 + (i64)blk_of[g * va + bl] * ns1 + i];
}

// modified Gram-Schmidt of the ns2 vectors of every aggregate (one CTA per aggregate); a vector
// the projections reduce to rounding (relative 1e-12 or less) sets *bad
__global__ void __launch_bounds__(MG_THREADS) k_mg_orth2(int ns2, int E, double2* __restrict__ P2, int* __restrict__ bad) {
  __shared__ double sh[2 * 8];
  double2* Pg = P2 + (i64)blockIdx.x * ns2 * E;
  for (int k = 0; k < ns2; ++k) {
    double2* wk = Pg + (i64)k * E;
    double n0[1] = {0.0};
    for (int e = threadIdx.x; e < E; e += blockDim.x) n0[0] += wk[e].x * wk[e].x + wk[e].y * wk[e].y;
    cta_sum<1>(n0, sh);
    for (int j = 0; j < k; ++j) {
      const double2* uj = Pg + (i64)j * E;
      double v[2] = {0.0, 0.0};
      for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const double2 a = uj[e], b = wk[e];
        v[0] += a.x * b.x + a.y * b.y;
        v[1] += a.x * b.y - a.y * b.x;
      }
      cta_sum<2>(v, sh);
      for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const double2 a = uj[e];
        double2 b = wk[e];
        b.x -= v[0] * a.x - v[1] * a.y;
        b.y -= v[0] * a.y + v[1] * a.x;
        wk[e] = b;
      }
    }
    double nn[1] = {0.0};
    for (int e = threadIdx.x; e < E; e += blockDim.x) nn[0] += wk[e].x * wk[e].x + wk[e].y * wk[e].y;
    cta_sum<1>(nn, sh);
    if (!(nn[0] > 1e-24 * n0[0])) {
      if (threadIdx.x == 0) atomicOr(bad, 1);
      return;  // uniform over the CTA
    }
    const double inv = 1.0 / sqrt(nn[0]);
    for (int e = threadIdx.x; e < E; e += blockDim.x) wk[e] = make_double2(wk[e].x * inv, wk[e].y * inv);
  }
}

struct AggGeom {
  int a[4];
};

// A2 = P2^+ A1 P2 from the stencil of A1 (one CTA per aggregate, one thread per (k2, k2')):
// the coupling of block b (local coordinates lc in its aggregate) to b' = nbr1[b][s1] adds to the
// self slot when b' lies in the same aggregate, else to slot s1 of the aggregate.
__global__ void __launch_bounds__(MG_THREADS)
    k_mg_galerkin(AggGeom ag, int ns1, int ns2, int va, int E, const double2* __restrict__ P2,
                  const double2* __restrict__ A1, const int* __restrict__ nbr1, const int* __restrict__ agg_of,
                  const int* __restrict__ loc_of, const int* __restrict__ blk_of, double2* __restrict__ A2) {
  const int g = blockIdx.x;
  for (int pr = threadIdx.x; pr < ns2 * ns2; pr += blockDim.x) {
    const int k2 = pr / ns2, kp = pr % ns2;
    double2 acc[DFL_SLOTS];
#pragma unroll
    for (int s = 0; s < DFL_SLOTS; ++s) acc[s] = make_double2(0.0, 0.0);
    for (int bl = 0; bl < va; ++bl) {
      const int b = blk_of[g * va + bl];
      int lc[4], u = bl;
      for (int mu = 3; mu >= 0; --mu) {
        lc[mu] = u % ag.a[mu];
        u /= ag.a[mu];
      }
      const double2* pg = P2 + ((i64)g * ns2 + k2) * E + bl * ns1;
#pragma unroll
      for (int s1 = 0; s1 < DFL_SLOTS; ++s1) {
        const int bp = nbr1[b * DFL_SLOTS + s1];
        const double2* pp = P2 + ((i64)agg_of[bp] * ns2 + kp) * E + loc_of[bp] * ns1;
        const double2* ab = A1 + ((i64)b * DFL_SLOTS + s1) * ns1 * ns1;
        double re = 0.0, im = 0.0;
        for (int i = 0; i < ns1; ++i) {
          double tr = 0.0, ti = 0.0;  // (A1 p')_i
          for (int j = 0; j < ns1; ++j) {
            const double2 a = ab[i * ns1 + j], v = pp[j];
            tr += a.x * v.x - a.y * v.y;
            ti += a.x * v.y + a.y * v.x;
          }
          const double2 c = pg[i];
          re += c.x * tr + c.y * ti;  // conj(c) t
          im += c.x * ti - c.y * tr;
        }
        bool cross = false;
        if (s1 > 0) {
          const int mu = (s1 - 1) >> 1;
          cross = ((s1 - 1) & 1) == 0 ? lc[mu] == ag.a[mu] - 1 : lc[mu] == 0;
        }
        if (cross) {
          acc[s1].x += re;
          acc[s1].y += im;
        } else {
          acc[0].x += re;
          acc[0].y += im;
        }
      }
    }
#pragma unroll
    for (int s = 0; s < DFL_SLOTS; ++s) A2[(((i64)g * DFL_SLOTS + s) * ns2 + k2) * ns2 + kp] = acc[s];
  }
}

#define MTRY(x)                  \
  do {                           \
    qxd_status _s = (x);         \
    if (_s != QXD_OK) return _s; \
  } while (0)

struct CLevel {
  int nb, ns;
  const double2* A;
  const int* nbr;
  i64 n;
};

static qxd_status cmv(qxd_lattice* lat, const CLevel& L, const double2* x, const double2* f, double2* y) {
  k_mg_cmv<<<egrid(L.n), 256, 0, lat->stream>>>(L.nb, L.ns, L.A, L.nbr, x, f, y);
  QXD_CHECK_LAUNCH(lat, "k_mg_cmv");
  return QXD_OK;
}

// out[j] = <Q_j, v> for j < nq (nq <= MG_MAXM); deterministic (fixed chunks and order); part:
// MG_MAXM x MG_DOT_BLOCKS scratch slots
static qxd_status cdots(qxd_lattice* lat, double2* part, const double2* Q, i64 n, int nq, const double2* v,
                        double2* out) {
  i64 nb = (n + MG_DOT_CHUNK - 1) / MG_DOT_CHUNK;
  if (nb > MG_DOT_BLOCKS) nb = MG_DOT_BLOCKS;
  if (nb < 1) nb = 1;
  const i64 chunk = (n + nb - 1) / nb;
  k_mg_dots_part<<<dim3((unsigned)nb, (unsigned)nq), 256, 0, lat->stream>>>(Q, n, chunk, v, part);
  QXD_CHECK_LAUNCH(lat, "k_mg_dots_part");
  k_mg_dots_fin<<<nq, 32, 0, lat->stream>>>(part, (int)nb, out);
  QXD_CHECK_LAUNCH(lat, "k_mg_dots_fin");
  return QXD_OK;
}

typedef std::function<qxd_status(const double2*, double2*)> CPre;

// nsteps (flexible) GCR steps on A x = f from x = 0, restart every m; work Z, W: m vectors each,
// r: one vector; dots: m + 2 device slots.
static qxd_status gcr_fixed(qxd_lattice* lat, double2* part, const CLevel& L, const double2* f, double2* x, int nsteps,
                            int m, double2* Z, double2* W, double2* r, double2* dots, const CPre* pre) {
  const i64 n = L.n;
  cudaStream_t S = lat->stream;
  QXD_CUDA(lat, cudaMemsetAsync(x, 0, sizeof(double2) * n, S));
  QXD_CUDA(lat, cudaMemcpyAsync(r, f, sizeof(double2) * n, cudaMemcpyDeviceToDevice, S));
  for (int it = 0; it < nsteps; ++it) {
    const int k = it % m;
    double2 *zk = Z + (i64)k * n, *wk = W + (i64)k * n;
    if (pre)
      MTRY((*pre)(r, zk));
    else
      QXD_CUDA(lat, cudaMemcpyAsync(zk, r, sizeof(double2) * n, cudaMemcpyDeviceToDevice, S));
    MTRY(cmv(lat, L, zk, nullptr, wk));
    if (k > 0) {
      MTRY(cdots(lat, part, W, n, k, wk, dots));
      k_mg_orth<<<egrid(n), 256, 0, S>>>(n, k, dots, W, Z, wk, zk);
      QXD_CHECK_LAUNCH(lat, "k_mg_orth");
    }
    MTRY(cdots(lat, part, wk, n, 1, wk, dots + m));
    k_mg_scale<<<egrid(n), 256, 0, S>>>(n, dots + m, wk, zk);
    QXD_CHECK_LAUNCH(lat, "k_mg_scale");
    MTRY(cdots(lat, part, wk, n, 1, r, dots + m + 1));
    k_mg_axpy2<<<egrid(n), 256, 0, S>>>(n, dots + m + 1, zk, x, wk, r);
    QXD_CHECK_LAUNCH(lat, "k_mg_axpy2");
  }
  return QXD_OK;
}

// y = S1 f (add = false) or y += S1 f (add = true): nu MR steps on A1 from zero
static qxd_status mr_smooth(qxd_lattice* lat, MgState* s, const CLevel& L1, const double2* f, double2* y, bool add) {
  const i64 n = L1.n;
  double2* rho = s->w1 + (i64)(2 * s->m + 1) * n;
  double2* q = rho + n;
  double2* d = s->sc + 2 * (s->m + 2);
  if (!add) QXD_CUDA(lat, cudaMemsetAsync(y, 0, sizeof(double2) * n, lat->stream));
  QXD_CUDA(lat, cudaMemcpyAsync(rho, f, sizeof(double2) * n, cudaMemcpyDeviceToDevice, lat->stream));
  for (int i = 0; i < s->nu; ++i) {
    MTRY(cmv(lat, L1, rho, nullptr, q));
    MTRY(cdots(lat, s->part, q, n, 1, rho, d));
    MTRY(cdots(lat, s->part, q, n, 1, q, d + 1));
    k_mg_mr<<<egrid(n), 256, 0, lat->stream>>>(n, d, rho, q, y);
    QXD_CHECK_LAUNCH(lat, "k_mg_mr");
  }
  return QXD_OK;
}

static CLevel level1(qxd_lattice* lat) {
  DflState* d = (DflState*)lat->dfl;
  return CLevel{d->dg.nb, d->ns, d->A, d->nbr, (i64)d->dg.nb * d->ns};
}
static CLevel level2(MgState* s) { return CLevel{s->nb2, s->ns2, s->A2, s->nbr2, s->n2}; }

// T1 f -> y (level-1 vectors; y must not alias f)
static qxd_status two_grid(qxd_lattice* lat, MgState* s, const double2* f, double2* y) {
  const CLevel L1 = level1(lat), L2 = level2(s);
  const i64 n1 = s->n1, n2 = s->n2;
  double2* t = s->w1 + (i64)(2 * s->m + 3) * n1;
  double2* f2 = s->w2 + (i64)(2 * s->m + 1) * n2;
  double2* c2 = f2 + n2;
  MTRY(mr_smooth(lat, s, L1, f, y, false));
  MTRY(cmv(lat, L1, y, f, t));  // t = f - A1 y
  k_mg_restrict2<<<(s->nb2 * s->ns2 + 255) / 256, 256, 0, lat->stream>>>(s->nb2, s->ns2, s->E, s->ns1, s->va, s->P2,
                                                                         s->blk_of, t, f2);
  QXD_CHECK_LAUNCH(lat, "k_mg_restrict2");
  MTRY(gcr_fixed(lat, s->part, L2, f2, c2, s->n2s, s->m, s->w2, s->w2 + (i64)s->m * n2, s->w2 + (i64)2 * s->m * n2,
                 s->sc + (s->m + 2), nullptr));
  k_mg_prolong2<<<(int)((n1 + 255) / 256), 256, 0, lat->stream>>>(s->nb1, s->ns1, s->ns2, s->E, s->P2, s->agg_of,
                                                                  s->loc_of, c2, y);
  QXD_CHECK_LAUNCH(lat, "k_mg_prolong2");
  MTRY(cmv(lat, L1, y, f, t));
  return mr_smooth(lat, s, L1, t, y, true);
}

// K1 f -> x (level-1 vectors)
static qxd_status level1_solve(qxd_lattice* lat, MgState* s, const double2* f, double2* x) {
  const CLevel L1 = level1(lat);
  const i64 n1 = s->n1;
  CPre pre = [lat, s](const double2* r, double2* z) { return two_grid(lat, s, r, z); };
  return gcr_fixed(lat, s->part, L1, f, x, s->n1s, s->m, s->w1, s->w1 + (i64)s->m * n1, s->w1 + (i64)2 * s->m * n1, s->sc,
                   &pre);
}

// K1 from the work vector f1 into c1, replayed from a CUDA graph captured on first use.  The
// capture runs on a private non-blocking stream (capture is refused on the legacy default stream)
// and only records; every replay runs on the lattice stream, after the work already queued there.
static qxd_status k1_run(qxd_lattice* lat, MgState* s) {
  double2* f1 = s->w1 + (i64)(2 * s->m + 4) * s->n1;
  double2* c1 = f1 + s->n1;
  if (!s->k1_exec) {
    if (!s->side) QXD_CUDA(lat, cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
    const cudaStream_t saved = lat->stream;
    const i64 l0 = lat->launches;
    QXD_CUDA(lat, cudaStreamBeginCapture(s->side, cudaStreamCaptureModeThreadLocal));
    lat->stream = s->side;
    const qxd_status st = level1_solve(lat, s, f1, c1);
    lat->stream = saved;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->side, &graph);
    if (st == QXD_OK && e == cudaSuccess) e = cudaGraphInstantiate(&s->k1_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    s->k1_launches = lat->launches - l0;
    lat->launches = l0;
    if (st != QXD_OK) return st;
    if (e != cudaSuccess) {
      s->k1_exec = nullptr;
      return cuda_fail(lat, e, "CUDA graph of the level-1 solve");
    }
  }
  QXD_CUDA(lat, cudaGraphLaunch(s->k1_exec, lat->stream));
  lat->launches += s->k1_launches;
  s->coarse_calls += 1;
  return QXD_OK;
}

// the fine preconditioner on FP32 full fields; scratch: work slots 58 and 59
qxd_status mg_precond32(qxd_lattice* lat, const SapSpec& sap, const float4* r, float4* z) {
  if (!mg_ready(lat)) return fail(lat, QXD_ESTATE, "multigrid not set up on the current deflation subspace (qxd_mg_setup)");
  MgState* s = (MgState*)lat->mg;
  DflState* d = (DflState*)lat->dfl;
  const i64 sv = lat->sv, n4 = 12 * sv;
  const size_t fb = sizeof(float4) * n4;
  float4 *dz, *t;
  MTRY(ensure_work(lat, 58, fb, (void**)&dz));
  MTRY(ensure_work(lat, 59, fb, (void**)&t));
  double2* f1 = s->w1 + (i64)(2 * s->m + 4) * s->n1;
  double2* c1 = f1 + s->n1;
  const int nt = dfl_threads(d->dg);
  auto residual = [&]() -> qxd_status {  // t = r - D z
    MTRY(hop32(lat, 0, EPI_DFULL, 0, z + 6 * sv, z, dz, 0.f));
    MTRY(hop32(lat, 1, EPI_DFULL, 0, z, z + 6 * sv, dz + 6 * sv, 0.f));
    MTRY(blas_copy(lat, t, r, fb));
    return blas_axpy_32(lat, -1.0f, dz, t, n4);
  };
  const float4* rc = r;
  if (s->ncy_pre > 0) {
    MTRY(sap32(lat, sap.block, s->ncy_pre, sap.nmr, r, z));
    MTRY(residual());
    rc = t;
  }
  k_dfl_restrict<<<d->dg.nb, nt, 0, lat->stream>>>(lat->g, d->dg, d->ns, d->basis32, rc, f1);
  QXD_CHECK_LAUNCH(lat, "k_dfl_restrict");
  MTRY(k1_run(lat, s));
  k_dfl_prolong<<<d->dg.nb, nt, 0, lat->stream>>>(lat->g, d->dg, d->ns, d->basis32, c1, dz);
  QXD_CHECK_LAUNCH(lat, "k_dfl_prolong");
  if (s->ncy_pre > 0)
    MTRY(blas_axpy_32(lat, 1.0f, dz, z, n4));
  else
    MTRY(blas_copy(lat, z, dz, fb));
  MTRY(residual());
  MTRY(sap32(lat, sap.block, sap.ncy, sap.nmr, t, dz));
  return blas_axpy_32(lat, 1.0f, dz, z, n4);
}

static qxd_status mg_check_params(qxd_lattice* lat, const qxd_mg_params* p) {
  if (!p) return fail(lat, QXD_EINVAL, "null argument");
  if (p->version != QXD_MG_VERSION) return fail(lat, QXD_EINVAL, "qxd_mg_params.version must be QXD_MG_VERSION");
  if (p->ns2 < 1 || p->ns2 > MG_MAXNS2) return fail(lat, QXD_EINVAL, "ns2 must be 1..32");
  if (p->nu < 0 || p->nu > 16) return fail(lat, QXD_EINVAL, "nu must be 0..16");
  if (p->n1 < 1 || p->n1 > 64) return fail(lat, QXD_EINVAL, "n1 must be 1..64");
  if (p->n2 < 1 || p->n2 > 256) return fail(lat, QXD_EINVAL, "n2 must be 1..256");
  if (p->m < 1 || p->m > MG_MAXM) return fail(lat, QXD_EINVAL, "m must be 1..16");
  if (p->ncy_pre < 0 || p->ncy_pre > 8) return fail(lat, QXD_EINVAL, "ncy_pre must be 0..8");
  return QXD_OK;
}

// host tables of the aggregation; EINVAL when the aggregates do not form a nearest-neighbour grid
static qxd_status mg_tables(qxd_lattice* lat, const DflState* d, const int a[4], MgState* s, std::vector<int>& agg_of,
                            std::vector<int>& loc_of, std::vector<int>& blk_of) {
  const DflGeom& dg = d->dg;
  s->va = 1;
  s->nb2 = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (a[mu] < 1 || dg.n[mu] % a[mu]) return fail(lat, QXD_EINVAL, "aggregate extents must divide the deflation block grid");
    s->agg[mu] = a[mu];
    s->n2g[mu] = dg.n[mu] / a[mu];
    s->va *= a[mu];
    s->nb2 *= s->n2g[mu];
  }
  s->nb1 = dg.nb;
  s->ns1 = d->ns;
  s->E = s->va * s->ns1;
  if (s->E > 4096) return fail(lat, QXD_EINVAL, "an aggregate may hold at most 4096 level-1 entries");
  agg_of.assign(dg.nb, 0);
  loc_of.assign(dg.nb, 0);
  blk_of.assign((size_t)s->nb2 * s->va, 0);
  for (int b = 0; b < dg.nb; ++b) {
    int kb[4], kg[4], lc[4];
    block_coords(dg, b, kb);
    for (int mu = 0; mu < 4; ++mu) {
      kg[mu] = kb[mu] / a[mu];
      lc[mu] = kb[mu] % a[mu];
    }
    const int g = ((kg[0] * s->n2g[1] + kg[1]) * s->n2g[2] + kg[2]) * s->n2g[3] + kg[3];
    const int l = ((lc[0] * a[1] + lc[1]) * a[2] + lc[2]) * a[3] + lc[3];
    agg_of[b] = g;
    loc_of[b] = l;
    blk_of[(size_t)g * s->va + l] = b;
  }
  // the aggregate neighbour table, checked against every face block
  s->hnbr2.assign((size_t)s->nb2 * DFL_SLOTS, -1);
  for (int b = 0; b < dg.nb; ++b) {
    const int g = agg_of[b], l = loc_of[b];
    int lc[4], u = l;
    for (int mu = 3; mu >= 0; --mu) {
      lc[mu] = u % a[mu];
      u /= a[mu];
    }
    s->hnbr2[(size_t)g * DFL_SLOTS] = g;
    for (int s1 = 1; s1 < DFL_SLOTS; ++s1) {
      const int mu = (s1 - 1) >> 1;
      const bool fwd = ((s1 - 1) & 1) == 0;
      const bool cross = fwd ? lc[mu] == a[mu] - 1 : lc[mu] == 0;
      const int gp = agg_of[d->hnbr[(size_t)b * DFL_SLOTS + s1]];
      if (!cross) {
        if (gp != g) return fail(lat, QXD_EINVAL, "aggregation: an interior step leaves the aggregate");
        continue;
      }
      int& e = s->hnbr2[(size_t)g * DFL_SLOTS + s1];
      if (e >= 0 && e != gp)
        return fail(lat, QXD_EINVAL,
                    "aggregation: the face blocks of an aggregate reach different aggregates (with C*, the x shift must be a "
                    "whole number of aggregates)");
      e = gp;
    }
  }
  return QXD_OK;
}

}  // namespace qxd

using namespace qxd;

extern "C" {

qxd_status qxd_mg_setup(qxd_lattice* lat, const qxd_mg_params* p, const double* vectors, int on_device) {
  QXD_TRACE();
  if (!lat) return QXD_EINVAL;
  MTRY(mg_check_params(lat, p));
  if (!vectors) return fail(lat, QXD_EINVAL, "null argument");
  if (!dfl_ready(lat)) return fail(lat, QXD_ESTATE, "multigrid needs a deflation subspace on the current field (qxd_dfl_setup)");
  DflState* d = (DflState*)lat->dfl;
  if (lat->mg) {
    lat->mg_release(lat->mg);
    lat->mg = nullptr;
  }
  MgState* s = new MgState();
  auto bail = [&](qxd_status st) {
    mg_release(s);
    return st;
  };
  std::vector<int> agg_of, loc_of, blk_of;
  {
    qxd_status st = mg_tables(lat, d, p->agg, s, agg_of, loc_of, blk_of);
    if (st) return bail(st);
  }
  s->ns2 = p->ns2;
  s->nu = p->nu;
  s->n1s = p->n1;
  s->n2s = p->n2;
  s->m = p->m;
  s->ncy_pre = p->ncy_pre;
  s->n1 = (i64)s->nb1 * s->ns1;
  s->n2 = (i64)s->nb2 * s->ns2;
  if (s->ns2 > s->E) return bail(fail(lat, QXD_EINVAL, "ns2 exceeds the entries of an aggregate"));
  bool ok = cudaMalloc(&s->P2, sizeof(double2) * (size_t)s->nb2 * s->ns2 * s->E) == cudaSuccess &&
            cudaMalloc(&s->A2, sizeof(double2) * (size_t)s->nb2 * DFL_SLOTS * s->ns2 * s->ns2) == cudaSuccess &&
            cudaMalloc(&s->nbr2, sizeof(int) * (size_t)s->nb2 * DFL_SLOTS) == cudaSuccess &&
            cudaMalloc(&s->agg_of, sizeof(int) * s->nb1) == cudaSuccess &&
            cudaMalloc(&s->loc_of, sizeof(int) * s->nb1) == cudaSuccess &&
            cudaMalloc(&s->blk_of, sizeof(int) * blk_of.size()) == cudaSuccess &&
            cudaMalloc(&s->w1, sizeof(double2) * (size_t)(2 * s->m + 6) * s->n1) == cudaSuccess &&
            cudaMalloc(&s->w2, sizeof(double2) * (size_t)(2 * s->m + 3) * s->n2) == cudaSuccess &&
            cudaMalloc(&s->sc, sizeof(double2) * (size_t)(2 * (s->m + 2) + 2)) == cudaSuccess &&
            cudaMalloc(&s->part, sizeof(double2) * (size_t)MG_MAXM * MG_DOT_BLOCKS) == cudaSuccess;
  if (!ok) return bail(fail(lat, QXD_ENOMEM, "multigrid allocation failed"));
  cudaStream_t S = lat->stream;
  if (cudaMemcpyAsync(s->nbr2, s->hnbr2.data(), sizeof(int) * s->hnbr2.size(), cudaMemcpyHostToDevice, S) != cudaSuccess ||
      cudaMemcpyAsync(s->agg_of, agg_of.data(), sizeof(int) * s->nb1, cudaMemcpyHostToDevice, S) != cudaSuccess ||
      cudaMemcpyAsync(s->loc_of, loc_of.data(), sizeof(int) * s->nb1, cudaMemcpyHostToDevice, S) != cudaSuccess ||
      cudaMemcpyAsync(s->blk_of, blk_of.data(), sizeof(int) * blk_of.size(), cudaMemcpyHostToDevice, S) != cudaSuccess ||
      cudaMemsetAsync(s->sc, 0, sizeof(double2) * (size_t)(2 * (s->m + 2) + 2), S) != cudaSuccess)
    return bail(fail(lat, QXD_ECUDA, "mg_setup: table upload"));
  // the caller's level-2 vectors [ns2][n1] complex
  const double2* V = (const double2*)vectors;
  const size_t vbytes = sizeof(double2) * (size_t)s->ns2 * s->n1;
  if (!on_device) {
    void* bi = nullptr;
    qxd_status st = ensure_work(lat, 26, vbytes, &bi);
    if (st) return bail(st);
    if (cudaMemcpyAsync(bi, vectors, vbytes, cudaMemcpyHostToDevice, S) != cudaSuccess)
      return bail(fail(lat, QXD_ECUDA, "mg_setup: copy of the vectors"));
    V = (const double2*)bi;
  }
  const i64 np2 = (i64)s->nb2 * s->ns2 * s->E;
  k_mg_gather2<<<(int)((np2 + 255) / 256), 256, 0, S>>>(s->nb2, s->ns2, s->E, s->ns1, s->va, s->blk_of, s->n1, V, s->P2);
  if (cudaGetLastError() != cudaSuccess) return bail(fail(lat, QXD_ECUDA, "k_mg_gather2 launch"));
  int* bad;
  {
    qxd_status st = ensure_work(lat, 30, sizeof(int), (void**)&bad);
    if (st) return bail(st);
  }
  cudaMemsetAsync(bad, 0, sizeof(int), S);
  k_mg_orth2<<<s->nb2, MG_THREADS, 0, S>>>(s->ns2, s->E, s->P2, bad);
  if (cudaGetLastError() != cudaSuccess) return bail(fail(lat, QXD_ECUDA, "k_mg_orth2 launch"));
  int hbad = 0;
  cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, S);
  if (cudaStreamSynchronize(S) != cudaSuccess) return bail(fail(lat, QXD_ECUDA, "mg_setup"));
  if (hbad) return bail(fail(lat, QXD_EINVAL, "level-2 vectors are linearly dependent on some aggregate"));
  AggGeom ag;
  for (int mu = 0; mu < 4; ++mu) ag.a[mu] = s->agg[mu];
  const int gth = std::min(MG_THREADS, (s->ns2 * s->ns2 + 31) / 32 * 32);
  k_mg_galerkin<<<s->nb2, gth, 0, S>>>(ag, s->ns1, s->ns2, s->va, s->E, s->P2, d->A, d->nbr, s->agg_of, s->loc_of,
                                              s->blk_of, s->A2);
  if (cudaGetLastError() != cudaSuccess) return bail(fail(lat, QXD_ECUDA, "k_mg_galerkin launch"));
  lat->launches += 3;
  if (cudaStreamSynchronize(S) != cudaSuccess) return bail(fail(lat, QXD_ECUDA, "mg_setup"));
  s->dfl_gen = d->gen;
  lat->mg = s;
  lat->mg_release = mg_release;
  return QXD_OK;
}

qxd_status qxd_mg_generate(qxd_lattice* lat, int ns2, int n_it, int k, const double* start, double* out, int on_device) {
  QXD_TRACE();
  if (!lat) return QXD_EINVAL;
  if (!start || !out) return fail(lat, QXD_EINVAL, "null argument");
  if (ns2 < 1 || n_it < 0 || k < 1 || k > 256) return fail(lat, QXD_EINVAL, "ns2 >= 1, n_it >= 0, 1 <= k <= 256");
  if (!dfl_ready(lat)) return fail(lat, QXD_ESTATE, "mg_generate needs a deflation subspace on the current field");
  const CLevel L1 = level1(lat);
  const i64 n = L1.n;
  const int m = MG_MAXM;
  const size_t vb = sizeof(double2) * n;
  double2 *w, *sc;
  // scratch: API slot 24 (vectors), 25 (scalars, then the inner-product partials)
  MTRY(ensure_work(lat, 24, vb * (2 * m + 3), (void**)&w));
  MTRY(ensure_work(lat, 25, sizeof(double2) * (m + 2 + MG_MAXM * MG_DOT_BLOCKS), (void**)&sc));
  double2* part = sc + m + 2;
  double2 *v = w + (i64)(2 * m + 1) * n, *x = v + n;
  cudaStream_t S = lat->stream;
  for (int j = 0; j < ns2; ++j) {
    const double2* src = (const double2*)start + (i64)j * n;
    double2* dst = (double2*)out + (i64)j * n;
    QXD_CUDA(lat, cudaMemcpyAsync(v, src, vb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, S));
    MTRY(cdots(lat, part, v, n, 1, v, sc));
    k_mg_scale1<<<egrid(n), 256, 0, S>>>(n, sc, v);
    QXD_CHECK_LAUNCH(lat, "k_mg_scale1");
    for (int it = 0; it < n_it; ++it) {
      MTRY(gcr_fixed(lat, part, L1, v, x, k, m, w, w + (i64)m * n, w + (i64)2 * m * n, sc, nullptr));
      MTRY(cdots(lat, part, x, n, 1, x, sc + m));
      k_mg_scale1<<<egrid(n), 256, 0, S>>>(n, sc + m, x);
      QXD_CHECK_LAUNCH(lat, "k_mg_scale1");
      std::swap(v, x);
    }
    QXD_CUDA(lat, cudaMemcpyAsync(dst, v, vb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, S));
    if (!on_device) QXD_CUDA(lat, cudaStreamSynchronize(S));
  }
  QXD_CUDA(lat, cudaStreamSynchronize(S));
  return QXD_OK;
}

qxd_status qxd_mg_get_coarse(qxd_lattice* lat, double* A2, int* nbr2) {
  QXD_TRACE();
  if (!lat) return QXD_EINVAL;
  if (!lat->mg) return fail(lat, QXD_ESTATE, "multigrid not set up");
  if (!A2 || !nbr2) return fail(lat, QXD_EINVAL, "null argument");
  MgState* s = (MgState*)lat->mg;
  const size_t ab = sizeof(double2) * (size_t)s->nb2 * DFL_SLOTS * s->ns2 * s->ns2;
  QXD_CUDA(lat, cudaMemcpyAsync(A2, s->A2, ab, cudaMemcpyDeviceToHost, lat->stream));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  std::memcpy(nbr2, s->hnbr2.data(), sizeof(int) * s->hnbr2.size());
  return QXD_OK;
}

qxd_status qxd_mg_info(qxd_lattice* lat, int* nb2, int* ns2, int64_t* level1_solves) {
  if (!lat) return QXD_EINVAL;
  if (!lat->mg) return fail(lat, QXD_ESTATE, "multigrid not set up");
  MgState* s = (MgState*)lat->mg;
  if (nb2) *nb2 = s->nb2;
  if (ns2) *ns2 = s->ns2;
  if (level1_solves) *level1_solves = s->coarse_calls;
  return QXD_OK;
}

qxd_status qxd_mg_apply_level1(qxd_lattice* lat, double* out, const double* in, int on_device) {
  QXD_TRACE();
  if (!lat) return QXD_EINVAL;
  if (!out || !in) return fail(lat, QXD_EINVAL, "null argument");
  if (!mg_ready(lat)) return fail(lat, QXD_ESTATE, "multigrid not set up on the current deflation subspace");
  MgState* s = (MgState*)lat->mg;
  const size_t vb = sizeof(double2) * s->n1;
  double2* f1 = s->w1 + (i64)(2 * s->m + 4) * s->n1;
  double2* c1 = f1 + s->n1;
  cudaStream_t S = lat->stream;
  QXD_CUDA(lat, cudaMemcpyAsync(f1, in, vb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, S));
  MTRY(k1_run(lat, s));
  QXD_CUDA(lat, cudaMemcpyAsync(out, c1, vb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, S));
  QXD_CUDA(lat, cudaStreamSynchronize(S));
  return QXD_OK;
}

qxd_status qxd_mg_precond(qxd_lattice* lat, double* out, const double* in, const int sap_block[4], int ncy, int nmr,
                          int on_device) {
  QXD_TRACE();
  if (!lat) return QXD_EINVAL;
  if (!out || !in || !sap_block) return fail(lat, QXD_EINVAL, "null argument");
  if (ncy < 1 || nmr < 1) return fail(lat, QXD_EINVAL, "ncy and nmr must be >= 1");
  if (!lat->have_clover) return fail(lat, QXD_ESTATE, "mg_precond before build_clover");
  MTRY(sap_check(lat, sap_block));
  if (!mg_ready(lat)) return fail(lat, QXD_ESTATE, "multigrid not set up on the current deflation subspace");
  const i64 sv = lat->sv;
  const size_t vb = sizeof(double) * 24 * lat->V;
  double2 *f64, *g64;
  float4 *a32, *b32;
  void *bi = nullptr, *bo = nullptr;
  MTRY(ensure_work(lat, 24, sizeof(double2) * 24 * sv, (void**)&f64));
  MTRY(ensure_work(lat, 25, sizeof(double2) * 24 * sv, (void**)&g64));
  MTRY(ensure_work(lat, 43, sizeof(float4) * 12 * sv, (void**)&a32));
  MTRY(ensure_work(lat, 44, sizeof(float4) * 12 * sv, (void**)&b32));
  const double* src = in;
  if (!on_device) {
    MTRY(ensure_work(lat, 26, vb, &bi));
    MTRY(ensure_work(lat, 27, vb, &bo));
    QXD_CUDA(lat, cudaMemcpyAsync(bi, in, vb, cudaMemcpyHostToDevice, lat->stream));
    src = (const double*)bi;
  }
  SapSpec sp;
  for (int mu = 0; mu < 4; ++mu) sp.block[mu] = sap_block[mu];
  sp.ncy = ncy;
  sp.nmr = nmr;
  MTRY(pack_spinor64(lat, (const double2*)src, f64, 0));
  MTRY(f64_to_f32(lat, f64, a32, 12 * sv));
  MTRY(mg_precond32(lat, sp, a32, b32));
  MTRY(f32_to_f64(lat, b32, g64, 12 * sv));
  MTRY(unpack_spinor64(lat, g64, on_device ? (double2*)out : (double2*)bo, 0));
  if (!on_device) {
    QXD_CUDA(lat, cudaMemcpyAsync(out, bo, vb, cudaMemcpyDeviceToHost, lat->stream));
  }
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  return QXD_OK;
}

}  // extern "C"
