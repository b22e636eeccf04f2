// Flexible GCR on the full D in FP32 with a right preconditioner M (the learned network, the
// Schwarz alternating procedure, or none), with every coefficient kept on the device.
//
// Cycle of at most m steps, k = 0, 1, ...:
//   z_k = M r;  w_k = D z_k;
//   c_jk = <w'_j, w_k> / ||w'_j||^2 (j < k, one multi-dot);  w'_k = w_k - sum_j c_jk w'_j
//   (classical Gram-Schmidt, optionally repeated once more);  alpha_k = <w'_k, r> / ||w'_k||^2;
//   r -= alpha_k w'_k.
// With z'_k = z_k - sum_j c_jk z'_j (so that D z'_k = w'_k) the solution update of the cycle is
// sum_k alpha_k z'_k = Z (I + C)^-1 alpha: at the end of a cycle one thread solves the unit upper
// triangular system (I + C) beta = alpha and one pass adds sum_k beta_k z_k to y, so the z_k are
// never orthogonalised.  The host reads ||r||^2 only every `check_every` steps.
//
// Reductions: per-block FP64 partials (FP32 products per element), summed in block order by a
// second small kernel: deterministic for a given grid.
#include "qxd_internal.cuh"
#include "sap.cuh"
#include "reduce.cuh"

namespace qxd {

#define TRY_Q(x)                     \
  do {                               \
    qxd_status _s = (x);             \
    if (_s != QXD_OK) return _s;     \
  } while (0)

constexpr int FG_MAXM = 32;
constexpr int FG_BLOCK = 256;

struct FgScal {
  double c[FG_MAXM][2 * FG_MAXM];  // c[k][2 j + re/im] = c_jk
  double nw2[FG_MAXM];             // ||w'_k||^2
  double alpha[2 * FG_MAXM];       // alpha_k
  double beta[2 * FG_MAXM];        // (I + C)^-1 alpha
  double rn2;                      // ||r||^2
  double pad;
};

// part[(b * 2 FG_MAXM) + 2 j + {re, im}] = block b's share of <w_j, v>, for the rows
// j = 8 blockIdx.y .. + 7 (< k): many small blocks (16 FP32 accumulators per thread) keep enough
// loads in flight; v is read once per group of eight rows.  FP32 partial sums per thread over its
// few elements, FP64 block reduction.
constexpr int FG_MDOT_BLOCKS = 152 * 4;
constexpr int FG_ROWS = 8;
__global__ void __launch_bounds__(FG_BLOCK) k_fg_mdot(const float4* __restrict__ W, i64 fs, int k,
                                                     const float4* __restrict__ v, i64 n4, double* __restrict__ part) {
  const int j0 = blockIdx.y * FG_ROWS;
  float acc[2 * FG_ROWS];
#pragma unroll
  for (int j = 0; j < 2 * FG_ROWS; ++j) acc[j] = 0.f;
  for (i64 i = blockIdx.x * (i64)FG_BLOCK + threadIdx.x; i < n4; i += (i64)gridDim.x * FG_BLOCK) {
    const float4 b = v[i];
#pragma unroll
    for (int j = 0; j < FG_ROWS; ++j) {
      if (j0 + j < k) {
        const float4 a = W[(i64)(j0 + j) * fs + i];
        acc[2 * j] += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
        acc[2 * j + 1] += a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
      }
    }
  }
  __shared__ double sh[2 * FG_ROWS][FG_BLOCK / 32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 2 * FG_ROWS; ++j) {
    const double d = warp_sum((double)acc[j]);
    if (lane == 0) sh[j][wp] = d;
  }
  __syncthreads();
  if (threadIdx.x < 2 * FG_ROWS && j0 + (threadIdx.x >> 1) < k) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < FG_BLOCK / 32; ++q) t += sh[threadIdx.x][q];
    part[(i64)blockIdx.x * 2 * FG_MAXM + 2 * j0 + threadIdx.x] = t;
  }
}

// row j = blockIdx.x: d_j = sum_b part (block order); c_jk (+)= d_j / ||w'_j||^2
__global__ void __launch_bounds__(FG_BLOCK) k_fg_mdot_fin(const double* __restrict__ part, int nb, int k, int add,
                                                         FgScal* S) {
  const int j = blockIdx.x;
  double acc[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += FG_BLOCK) {
    acc[0] += part[(i64)b * 2 * FG_MAXM + 2 * j];
    acc[1] += part[(i64)b * 2 * FG_MAXM + 2 * j + 1];
  }
  block_sum<2, FG_BLOCK>(acc);
  if (threadIdx.x == 0) {
    const double n = S->nw2[j];
    S->c[k][2 * j] = (add ? S->c[k][2 * j] : 0.0) + acc[0] / n;
    S->c[k][2 * j + 1] = (add ? S->c[k][2 * j + 1] : 0.0) + acc[1] / n;
  }
}

// w_k -= sum_j c_j w_j with c_j the coefficients of this pass (cur: this pass's, minus the earlier
// ones when add); partials of ||w_k||^2 and <w_k, r>
__global__ void __launch_bounds__(FG_BLOCK) k_fg_orth(const float4* __restrict__ W, i64 fs, int k, float4* __restrict__ wk,
                                                     const float4* __restrict__ r, i64 n4, const double* __restrict__ cprev,
                                                     const FgScal* __restrict__ S, double* __restrict__ part) {
  __shared__ float2 cs[FG_MAXM];
  if (threadIdx.x < k) {
    const double pr = cprev ? cprev[2 * threadIdx.x] : 0.0, pi = cprev ? cprev[2 * threadIdx.x + 1] : 0.0;
    cs[threadIdx.x] = make_float2((float)(S->c[k][2 * threadIdx.x] - pr), (float)(S->c[k][2 * threadIdx.x + 1] - pi));
  }
  __syncthreads();
  double acc[3] = {0.0, 0.0, 0.0};
  for (i64 i = blockIdx.x * (i64)FG_BLOCK + threadIdx.x; i < n4; i += (i64)gridDim.x * FG_BLOCK) {
    float4 a = wk[i];
#pragma unroll 8
    for (int j = 0; j < k; ++j) {  // unrolled: eight basis loads in flight
      const float4 u = W[(i64)j * fs + i];
      const float2 c = cs[j];
      a.x -= c.x * u.x - c.y * u.y;
      a.y -= c.x * u.y + c.y * u.x;
      a.z -= c.x * u.z - c.y * u.w;
      a.w -= c.x * u.w + c.y * u.z;
    }
    wk[i] = a;
    const float4 b = r[i];
    acc[0] += (double)(a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w);
    acc[1] += (double)(a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w);
    acc[2] += (double)(a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z);
  }
  block_sum<3, FG_BLOCK>(acc);
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) part[(i64)blockIdx.x * 3 + q] = acc[q];
}

// ||w'_k||^2 and alpha_k = <w'_k, r> / ||w'_k||^2
__global__ void __launch_bounds__(FG_BLOCK) k_fg_orth_fin(const double* __restrict__ part, int nb, int k, FgScal* S) {
  double acc[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += FG_BLOCK)
    for (int q = 0; q < 3; ++q) acc[q] += part[(i64)b * 3 + q];
  block_sum<3, FG_BLOCK>(acc);
  if (threadIdx.x == 0) {
    S->nw2[k] = acc[0];
    S->alpha[2 * k] = acc[1] / acc[0];
    S->alpha[2 * k + 1] = acc[2] / acc[0];
  }
}

// r -= alpha_k w'_k; partials of ||r||^2
__global__ void __launch_bounds__(FG_BLOCK) k_fg_update(const float4* __restrict__ wk, float4* __restrict__ r, i64 n4, int k,
                                                       const FgScal* __restrict__ S, double* __restrict__ part) {
  const float ar = (float)S->alpha[2 * k], ai = (float)S->alpha[2 * k + 1];
  double acc[1] = {0.0};
  for (i64 i = blockIdx.x * (i64)FG_BLOCK + threadIdx.x; i < n4; i += (i64)gridDim.x * FG_BLOCK) {
    const float4 u = wk[i];
    float4 v = r[i];
    v.x -= ar * u.x - ai * u.y;
    v.y -= ar * u.y + ai * u.x;
    v.z -= ar * u.z - ai * u.w;
    v.w -= ar * u.w + ai * u.z;
    r[i] = v;
    acc[0] += (double)(v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w);
  }
  block_sum<1, FG_BLOCK>(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

// partials of ||v||^2
__global__ void __launch_bounds__(FG_BLOCK) k_fg_norm2(const float4* __restrict__ v, i64 n4, double* __restrict__ part) {
  double acc[1] = {0.0};
  for (i64 i = blockIdx.x * (i64)FG_BLOCK + threadIdx.x; i < n4; i += (i64)gridDim.x * FG_BLOCK) {
    const float4 a = v[i];
    acc[0] += (double)(a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w);
  }
  block_sum<1, FG_BLOCK>(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

__global__ void __launch_bounds__(FG_BLOCK) k_fg_sum1(const double* __restrict__ part, int nb, double* out) {
  double acc[1] = {0.0};
  for (int b = threadIdx.x; b < nb; b += FG_BLOCK) acc[0] += part[b];
  block_sum<1, FG_BLOCK>(acc);
  if (threadIdx.x == 0) *out = acc[0];
}

// (I + C) beta = alpha for the first kk steps of the cycle (back substitution, one thread)
__global__ void k_fg_beta(int kk, FgScal* S) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int j = kk - 1; j >= 0; --j) {
    double br = S->alpha[2 * j], bi = S->alpha[2 * j + 1];
    for (int k = j + 1; k < kk; ++k) {
      const double cr = S->c[k][2 * j], ci = S->c[k][2 * j + 1], xr = S->beta[2 * k], xi = S->beta[2 * k + 1];
      br -= cr * xr - ci * xi;
      bi -= cr * xi + ci * xr;
    }
    S->beta[2 * j] = br;
    S->beta[2 * j + 1] = bi;
  }
}

// y += sum_k beta_k z_k
__global__ void __launch_bounds__(FG_BLOCK) k_fg_zsum(const float4* __restrict__ Z, i64 fs, int kk, float4* __restrict__ y,
                                                     i64 n4, const FgScal* __restrict__ S) {
  __shared__ float2 bs[FG_MAXM];
  if (threadIdx.x < kk) bs[threadIdx.x] = make_float2((float)S->beta[2 * threadIdx.x], (float)S->beta[2 * threadIdx.x + 1]);
  __syncthreads();
  for (i64 i = blockIdx.x * (i64)FG_BLOCK + threadIdx.x; i < n4; i += (i64)gridDim.x * FG_BLOCK) {
    float4 a = y[i];
#pragma unroll 8
    for (int k = 0; k < kk; ++k) {
      const float4 u = Z[(i64)k * fs + i];
      const float2 b = bs[k];
      a.x += b.x * u.x - b.y * u.y;
      a.y += b.x * u.y + b.y * u.x;
      a.z += b.x * u.z - b.y * u.w;
      a.w += b.x * u.w + b.y * u.z;
    }
    y[i] = a;
  }
}

qxd_status fgcr32(qxd_lattice* lat, qxd_net* net, const SapSpec* sap, int m, int reorth, const float4* rhs, float4* y,
                  double target, int maxiter, int check_every, int* iters) {
  if (m < 1 || m > FG_MAXM) return fail(lat, QXD_EINVAL, "gcr_restart must be 1..32");
  const i64 sv = lat->sv, n4 = 12 * sv;
  const size_t fb = sizeof(float4) * n4;
  cudaStream_t S = lat->stream;
  float4 *r, *Z;
  FgScal* sc;
  double* part;
  const int nb = (int)std::min<i64>((n4 + FG_BLOCK - 1) / FG_BLOCK, lat->red_blocks);
  qxd_status st;
  if ((st = ensure_work(lat, 29, fb, (void**)&r))) return st;
  if ((st = ensure_work(lat, 31, fb * 2 * m, (void**)&Z))) return st;
  if ((st = ensure_work(lat, 40, sizeof(FgScal) + sizeof(double) * ((size_t)2 * FG_MAXM * std::max(nb, FG_MDOT_BLOCKS) + 3 * nb),
                        (void**)&sc)))
    return st;
  part = (double*)(sc + 1);
  double* part3 = part + (size_t)2 * FG_MAXM * std::max(nb, FG_MDOT_BLOCKS);
  auto z = [&](int k) { return Z + (i64)k * n4; };
  auto w = [&](int k) { return Z + (i64)(m + k) * n4; };
  QXD_CUDA(lat, cudaMemcpyAsync(r, rhs, fb, cudaMemcpyDeviceToDevice, S));
  k_fg_norm2<<<nb, FG_BLOCK, 0, S>>>(r, n4, part3);
  QXD_CHECK_LAUNCH(lat, "k_fg_norm2");
  k_fg_sum1<<<1, FG_BLOCK, 0, S>>>(part3, nb, &sc->rn2);
  QXD_CHECK_LAUNCH(lat, "k_fg_sum1");
  double rn2 = 0.0;
  QXD_CUDA(lat, cudaMemcpyAsync(lat->hscal, &sc->rn2, sizeof(double), cudaMemcpyDeviceToHost, S));
  QXD_CUDA(lat, cudaStreamSynchronize(S));
  rn2 = lat->hscal[0];
  int it = 0, k = 0;
  const int every = check_every > 0 ? check_every : 1;
  bool done = !(std::sqrt(rn2) > target);
  while (!done && it < maxiter) {
    if (sap && sap->mg)
      TRY_Q(mg_precond32(lat, *sap, r, z(k)));
    else if (sap && sap->dfl)
      TRY_Q(dfl_precond32(lat, *sap, r, z(k)));
    else if (sap)
      TRY_Q(sap32(lat, sap->block, sap->ncy, sap->nmr, r, z(k)));
    else if (net)
      TRY_Q(net_apply32(net, r, z(k)));
    else
      QXD_CUDA(lat, cudaMemcpyAsync(z(k), r, fb, cudaMemcpyDeviceToDevice, S));
    TRY_Q(hop32(lat, 0, EPI_DFULL, 0, z(k) + 6 * sv, z(k), w(k), 0.f));
    TRY_Q(hop32(lat, 1, EPI_DFULL, 0, z(k), z(k) + 6 * sv, w(k) + 6 * sv, 0.f));
    for (int pass = 0; pass < (k > 0 ? reorth : 0); ++pass) {  // classical Gram-Schmidt, once or twice
      const int mb = (int)std::min<i64>((n4 + FG_BLOCK - 1) / FG_BLOCK, FG_MDOT_BLOCKS);
      k_fg_mdot<<<dim3(mb, (k + FG_ROWS - 1) / FG_ROWS), FG_BLOCK, 0, S>>>(w(0), n4, k, w(k), n4, part);
      QXD_CHECK_LAUNCH(lat, "k_fg_mdot");
      k_fg_mdot_fin<<<k, FG_BLOCK, 0, S>>>(part, mb, k, pass > 0, sc);
      QXD_CHECK_LAUNCH(lat, "k_fg_mdot_fin");
      // this pass subtracts only its own coefficients: on the second pass the first pass's were
      // saved in beta (free until the end of the cycle)
      if (pass == 0 && reorth > 1) {
        QXD_CUDA(lat, cudaMemcpyAsync(sc->beta, sc->c[k], sizeof(double) * 2 * k, cudaMemcpyDeviceToDevice, S));
      }
      k_fg_orth<<<nb, FG_BLOCK, 0, S>>>(w(0), n4, k, w(k), r, n4, pass > 0 ? sc->beta : nullptr, sc, part3);
      QXD_CHECK_LAUNCH(lat, "k_fg_orth");
    }
    if (k == 0 || reorth == 0) {
      k_fg_orth<<<nb, FG_BLOCK, 0, S>>>(w(0), n4, 0, w(k), r, n4, nullptr, sc, part3);  // norms only
      QXD_CHECK_LAUNCH(lat, "k_fg_orth");
    }
    k_fg_orth_fin<<<1, FG_BLOCK, 0, S>>>(part3, nb, k, sc);
    QXD_CHECK_LAUNCH(lat, "k_fg_orth_fin");
    k_fg_update<<<nb, FG_BLOCK, 0, S>>>(w(k), r, n4, k, sc, part3);
    QXD_CHECK_LAUNCH(lat, "k_fg_update");
    k_fg_sum1<<<1, FG_BLOCK, 0, S>>>(part3, nb, &sc->rn2);
    QXD_CHECK_LAUNCH(lat, "k_fg_sum1");
    ++it;
    ++k;
    const bool check = it % every == 0 || it >= maxiter;
    if (check) {
      QXD_CUDA(lat, cudaMemcpyAsync(lat->hscal, &sc->rn2, sizeof(double), cudaMemcpyDeviceToHost, S));
      QXD_CUDA(lat, cudaStreamSynchronize(S));
      rn2 = lat->hscal[0];
      if (!std::isfinite(rn2)) {  // y keeps the cycles completed before this one
        *iters = it;
        return fail(lat, QXD_ENOCONV, "non-finite residual in FGCR");
      }
      done = !(std::sqrt(rn2) > target);
    }
    if (k == m || done || it >= maxiter) {  // end of the cycle: y += Z (I + C)^-1 alpha
      k_fg_beta<<<1, 32, 0, S>>>(k, sc);
      QXD_CHECK_LAUNCH(lat, "k_fg_beta");
      k_fg_zsum<<<nb, FG_BLOCK, 0, S>>>(Z, n4, k, y, n4, sc);
      QXD_CHECK_LAUNCH(lat, "k_fg_zsum");
      k = 0;
    }
  }
  *iters = it;
  if (net) TRY_Q(net_check(net));
  return QXD_OK;
}

}  // namespace qxd
