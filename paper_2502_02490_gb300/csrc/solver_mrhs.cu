// Multi-right-hand-side solve of D psi_r = eta_r, r = 0..n-1 (e.g. the 12 spin-colour point
// sources of a propagator), in lock step.
//
// Outer: per right-hand side, the FP64 defect correction of the single-RHS solver (FP64 D and
// norms, Schur source and reconstruction in FP32).  Inner: BiCGStab on Dhat for all right-hand
// sides at once with FP32 vectors, its Dhat applications by the multi-RHS hop (one link and
// clover load per site serves every right-hand side; FP32, or 16-bit spinors, links and clover
// with per-site norms), its vector updates and FP64 reductions by the
// BiCGStab kernels launched over (site blocks x right-hand sides) with per-RHS scalars.  A
// right-hand side that reaches its inner target is frozen (SC_ACTIVE = 0) while the others go
// on; each gets its own FP32 reliable updates (recompute s, restart).
#include <chrono>
#include <cmath>
#include <vector>

#include "qxd_internal.cuh"

namespace qxd {

qxd_status apply_D64(qxd_lattice* lat, const double2* in, double2* out);

#define TRY(x)                   \
  do {                           \
    qxd_status _s = (x);         \
    if (_s != QXD_OK) return _s; \
  } while (0)

enum { MW_HALVES = 32, MW_R32 = 33, MW_R64 = 34, MW_T64 = 35, MW_RO = 36, MW_H16 = 46, MW_H16N = 47 };
enum { H_BH = 0, H_Y, H_X, H_R, H_RH, H_P, H_V, H_S, H_T, H_TMP, H_N };

// Dhat on the n right-hand sides listed in rhs (FP32, multi-RHS hop): out = Dhat in, tmp odd-half
// scratch
static qxd_status dhat_mr(qxd_lattice* lat, const float4* in, float4* out, float4* tmp, int n, i64 rs, const int* rhs) {
  TRY(hop32_mrhs(lat, 1, EPI_INV, 0, in, nullptr, tmp, 1.0f, n, rs, rhs));
  TRY(hop32_mrhs(lat, 0, EPI_DHAT2, 0, tmp, in, out, -0.25f, n, rs, rhs));
  return QXD_OK;
}

static qxd_status read_mr(qxd_lattice* lat, int n) {
  QXD_CUDA(lat, cudaMemcpyAsync(lat->mr_hscal, lat->mr_scal, sizeof(double) * SC_N * n, cudaMemcpyDeviceToHost,
                                lat->stream));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  return QXD_OK;
}

// Inner lock-step BiCGStab for the active right-hand sides (act[i]); targets per RHS.  With a
// 16-bit inner precision the Dhat applications read 16-bit copies of p and s (with per-site
// norms) that the vector kernels write as they update p and s, as in the single-RHS solver.
static qxd_status inner_mr(qxd_lattice* lat, float4* H, int n, int prec, const std::vector<char>& act,
                           const std::vector<double>& target, double delta, int maxiter, int check_every, int* iters,
                           int* nrel) {
  const i64 sv = lat->sv, n4 = 6 * sv, rs = n4;
  auto half = [&](int k, int i) { return H + ((i64)k * n + i) * n4; };
  float4 *bh = half(H_BH, 0), *y = half(H_Y, 0), *x = half(H_X, 0), *r = half(H_R, 0), *rh = half(H_RH, 0),
         *p = half(H_P, 0), *v = half(H_V, 0), *s = half(H_S, 0), *t = half(H_T, 0), *tmp = half(H_TMP, 0);
  const size_t all = sizeof(float4) * n4 * n;
  const bool low = prec == QXD_F16N || prec == QXD_BF16N;
  const int bf = prec == QXD_BF16N;
  uint2* h16 = nullptr;
  float* h16n = nullptr;
  if (low) {  // [P, S, T][rhs][6][sv] 16-bit values and [P, S, T][rhs][sv] norms
    TRY(ensure_work(lat, MW_H16, sizeof(uint2) * 3 * n4 * n, (void**)&h16));
    TRY(ensure_work(lat, MW_H16N, sizeof(float) * 3 * sv * n, (void**)&h16n));
  }
  uint2 *p16 = h16, *s16 = h16 ? h16 + n4 * n : nullptr, *t16 = h16 ? h16 + 2 * n4 * n : nullptr;
  float *p16n = h16n, *s16n = h16n ? h16n + sv * n : nullptr, *t16n = h16n ? h16n + 2 * sv * n : nullptr;
  std::vector<char> on(act);  // right-hand sides still iterating
  // out = Dhat in for every active right-hand side (FP32 out); a frozen one keeps its old out
  std::vector<int> live;
  auto dhat_all = [&](const float4* in32, const uint2* in16, const float* in16n, float4* out) -> qxd_status {
    if (!low) {
      live.clear();
      for (int i = 0; i < n; ++i)
        if (on[i]) live.push_back(i);
      return live.empty() ? QXD_OK : dhat_mr(lat, in32, out, tmp, (int)live.size(), rs, live.data());
    }
    TRY(hop16_mrhs(lat, bf, 1, EPI_INV, 0, in16, in16n, nullptr, nullptr, t16, t16n, nullptr, 1.0f, n));
    return hop16_mrhs(lat, bf, 0, EPI_DHAT2, 0, t16, t16n, in16, in16n, nullptr, nullptr, out, -0.25f, n);
  };
  Rhs R;
  R.nrhs = n;
  R.rs = rs;
  R.mr = true;
  R.r0 = 0;
  auto one = [&](int i) {
    Rhs q;
    q.nrhs = 1;
    q.rs = 0;
    q.mr = true;
    q.r0 = i;
    return q;
  };
  for (int i = 0; i < n; ++i) TRY(set_scalar_at(lat, lat->mr_scal + (i64)i * SC_N + SC_ACTIVE, on[i] ? 1.0 : 0.0));
  TRY(blas_zero(lat, x, all));
  TRY(blas_copy(lat, r, bh, all));
  TRY(blas_copy(lat, rh, r, all));
  TRY(blas_copy(lat, p, r, all));
  if (low)
    for (int i = 0; i < n; ++i) TRY(f32_to_n16(lat, half(H_P, i), p16 + (i64)i * n4, p16n + (i64)i * sv, bf));
  TRY(bicg_cdot(lat, rh, r, SC_RHO, R));
  TRY(bicg_cdot(lat, r, r, SC_RN, R));
  TRY(read_mr(lat, n));
  std::vector<double> rmax(n);
  int nact = 0;
  for (int i = 0; i < n; ++i) {
    rmax[i] = std::sqrt(lat->mr_hscal[(i64)i * SC_N + SC_RN]);
    if (on[i] && rmax[i] <= target[i]) {
      on[i] = 0;
      TRY(set_scalar_at(lat, lat->mr_scal + (i64)i * SC_N + SC_ACTIVE, 0.0));
    }
    nact += on[i];
  }
  int it = 0, rel = 0;
  // the vector kernels timed as one class; algorithmic bytes: FP32 vectors of 96 B per site and
  // RHS, 16-bit copies 52 B
  const double vb = 96.0 * (double)lat->Vh * n, cb16 = low ? 52.0 * (double)lat->Vh * n : 0.0;
  auto timed = [&](double bytes, auto&& launch) -> qxd_status {
    prof_begin(lat, KSTAT_MR_BLAS, bytes);
    const qxd_status st = launch();
    prof_end(lat);
    return st;
  };
  while (nact > 0 && it < maxiter) {
    TRY(dhat_all(p, p16, p16n, v));
    TRY(timed(2 * vb, [&] { return bicg_cdot(lat, rh, v, SC_RV, R); }));
    TRY(timed(3 * vb + cb16, [&] { return bicg_s(lat, r, v, s, s16, s16n, bf, R); }));
    TRY(dhat_all(s, s16, s16n, t));
    TRY(timed(2 * vb, [&] { return bicg_ts(lat, t, s, R); }));
    TRY(timed(7 * vb, [&] { return bicg_xr(lat, x, p, s, t, rh, r, R); }));
    TRY(timed(4 * vb + cb16, [&] { return bicg_p(lat, r, v, p, p16, p16n, bf, R); }));
    ++it;
    if (it % check_every) continue;
    TRY(read_mr(lat, n));
    for (int i = 0; i < n; ++i) {
      if (!on[i]) continue;
      const double rn2 = lat->mr_hscal[(i64)i * SC_N + SC_RN];
      if (!std::isfinite(rn2)) return fail(lat, QXD_ENOCONV, "non-finite residual in the multi-RHS BiCGStab");
      double rn = std::sqrt(rn2);
      if (rn > rmax[i]) rmax[i] = rn;
      if (rn < delta * rmax[i] || rn <= target[i]) {
        // reliable update of RHS i: fold x_i into y_i, recompute r_i = bh_i - Dhat32 y_i
        float4 *xi = half(H_X, i), *yi = half(H_Y, i), *ri = half(H_R, i), *vi = half(H_V, i), *ti = half(H_TMP, i);
        TRY(blas_axpy_32(lat, 1.0f, xi, yi, n4));
        TRY(blas_zero(lat, xi, sizeof(float4) * n4));
        TRY(hop32(lat, 1, EPI_INV, 0, yi, nullptr, ti, 1.0f));
        TRY(hop32(lat, 0, EPI_DHAT2, 0, ti, yi, vi, -0.25f));
        TRY(blas_copy(lat, ri, half(H_BH, i), sizeof(float4) * n4));
        TRY(blas_axpy_32(lat, -1.0f, vi, ri, n4));
        TRY(bicg_cdot(lat, ri, ri, SC_RN, one(i)));
        QXD_CUDA(lat, cudaMemcpyAsync(lat->mr_hscal + (i64)i * SC_N + SC_RN, lat->mr_scal + (i64)i * SC_N + SC_RN,
                                      sizeof(double), cudaMemcpyDeviceToHost, lat->stream));
        QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
        rn = std::sqrt(lat->mr_hscal[(i64)i * SC_N + SC_RN]);
        rmax[i] = rn;
        ++rel;
        if (rn <= target[i]) {
          on[i] = 0;
          --nact;
          TRY(set_scalar_at(lat, lat->mr_scal + (i64)i * SC_N + SC_ACTIVE, 0.0));
        } else {
          TRY(blas_copy(lat, half(H_RH, i), ri, sizeof(float4) * n4));
          TRY(bicg_copy(lat, ri, half(H_P, i), low ? p16 + (i64)i * n4 : nullptr, low ? p16n + (i64)i * sv : nullptr,
                        bf));
          TRY(bicg_cdot(lat, ri, ri, SC_RHO, one(i)));
        }
      }
    }
  }
  TRY(blas_axpy_32(lat, 1.0f, x, y, 6 * sv * n));
  *iters = it;
  *nrel = rel;
  return QXD_OK;
}

// x, b: n full FP64 fields [n][2][12][sv] (device, internal layout); info: n entries or null
qxd_status solve_mrhs(qxd_lattice* lat, double2* x, const double2* b, int n, const qxd_solve_params* prm,
                      qxd_solve_info* info) {
  auto t0 = std::chrono::steady_clock::now();
  const i64 sv = lat->sv, nh = 12 * sv, nf = 24 * sv;
  TRY(ensure_mrhs(lat, n));
  float4 *H, *r32;
  double2 *r64, *t64;
  TRY(ensure_work(lat, MW_HALVES, sizeof(float4) * 6 * sv * n * H_N, (void**)&H));
  TRY(ensure_work(lat, MW_R32, sizeof(float4) * 12 * sv, (void**)&r32));
  TRY(ensure_work(lat, MW_R64, sizeof(double2) * nf, (void**)&r64));
  TRY(ensure_work(lat, MW_T64, sizeof(double2) * nf, (void**)&t64));
  auto half = [&](int k, int i) { return H + ((i64)k * n + i) * 6 * sv; };
  std::vector<double> bnorm(n), rel(n, 1.0), target(n);
  std::vector<char> done(n, 0);
  for (int i = 0; i < n; ++i) {
    double v;
    TRY(blas_norm2_64(lat, b + (i64)i * nf, nf, SC_TMP0));
    TRY(read_scalars(lat, SC_TMP0, 1, &v));
    bnorm[i] = std::sqrt(v);
    if (bnorm[i] == 0.0) {
      done[i] = 1;
      rel[i] = 0.0;
    }
  }
  TRY(blas_zero(lat, x, sizeof(double2) * nf * n));
  int total = 0, outer = 0, nrel = 0;
  const int max_outer = prm->max_outer > 0 ? prm->max_outer : 20;
  for (; outer <= max_outer; ++outer) {
    std::vector<char> act(n, 0);
    int nact = 0;
    for (int i = 0; i < n; ++i) {
      if (done[i]) continue;
      const double2* bi = b + (i64)i * nf;
      double2* xi = x + (i64)i * nf;
      if (outer == 0) {
        TRY(blas_copy(lat, r64, bi, sizeof(double2) * nf));
      } else {
        TRY(apply_D64(lat, xi, t64));
        TRY(blas_copy(lat, r64, bi, sizeof(double2) * nf));
        TRY(blas_axpy_64(lat, -1.0, 0.0, t64, r64, nf));
      }
      double rn2;
      TRY(blas_norm2_64(lat, r64, nf, SC_TMP0));
      TRY(read_scalars(lat, SC_TMP0, 1, &rn2));
      rel[i] = std::sqrt(rn2) / bnorm[i];
      if (!std::isfinite(rel[i])) return fail(lat, QXD_ENOCONV, "non-finite residual");
      if (rel[i] <= prm->tol) {
        done[i] = 1;
        continue;
      }
      // Schur source of the correction in FP32; keep the FP32 residual's odd half for the
      // reconstruction (H_TMP of RHS i holds it until the inner solve's scratch use)
      TRY(f64_to_f32(lat, r64, r32, 12 * sv));
      TRY(clover_apply32(lat, 1, 1, r32 + 6 * sv, half(H_T, i)));
      TRY(hop32(lat, 0, EPI_XPAY, 0, half(H_T, i), r32, half(H_BH, i), 0.5f));
      TRY(blas_copy(lat, half(H_S, i), r32 + 6 * sv, sizeof(float4) * 6 * sv));  // r_o saved in H_S
      target[i] = std::max(prm->inner_tol * std::sqrt(rn2), 0.5 * prm->tol * bnorm[i]);
      act[i] = 1;
      ++nact;
    }
    if (nact == 0) break;
    if (outer == max_outer || total >= prm->maxiter) break;
    // the saved odd residuals move out of H_S (the inner solve reuses it)
    float4* ro_save;
    TRY(ensure_work(lat, MW_RO, sizeof(float4) * 6 * sv * n, (void**)&ro_save));
    for (int i = 0; i < n; ++i)
      if (act[i]) TRY(blas_copy(lat, ro_save + (i64)i * 6 * sv, half(H_S, i), sizeof(float4) * 6 * sv));
    for (int i = 0; i < n; ++i)
      if (!act[i]) TRY(blas_zero(lat, half(H_BH, i), sizeof(float4) * 6 * sv));
    TRY(blas_zero(lat, half(H_Y, 0), sizeof(float4) * 6 * sv * n));
    int it = 0, nr = 0;
    TRY(inner_mr(lat, H, n, prm->inner_prec, act, target, prm->reliable_delta, prm->maxiter - total,
                 prm->check_every > 0 ? prm->check_every : 1, &it, &nr));
    if (prm->inner_prec == QXD_F32) TRY(mrhs_tile_status(lat));
    total += it;
    nrel += nr;
    // reconstruct each corrected RHS: x_e += y;  x_o += A_oo^-1 (r_o + 1/2 H_oe y)
    for (int i = 0; i < n; ++i) {
      if (!act[i]) continue;
      double2* xi = x + (i64)i * nf;
      TRY(hop32(lat, 1, EPI_INVXPAY, 0, half(H_Y, i), ro_save + (i64)i * 6 * sv, half(H_T, i), 0.5f));
      TRY(blas_acc_f32_into_f64(lat, half(H_Y, i), xi, 6 * sv));
      TRY(blas_acc_f32_into_f64(lat, half(H_T, i), xi + nh, 6 * sv));
    }
  }
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  bool ok = true;
  for (int i = 0; i < n; ++i) {
    ok = ok && done[i];
    if (info) {
      info[i].iters_inner = total;
      info[i].iters_outer = outer;
      info[i].reliable_updates = nrel;
      info[i].true_rel_res = rel[i];
      info[i].seconds = secs;
      info[i].status = done[i] ? QXD_OK : QXD_ENOCONV;
    }
  }
  if (!ok) return fail(lat, QXD_ENOCONV, "some right-hand side did not reach the tolerance");
  return QXD_OK;
}

}  // namespace qxd
