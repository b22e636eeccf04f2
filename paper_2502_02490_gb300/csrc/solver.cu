// Solvers for D psi = eta on the even-odd preconditioned system.
//
//   Dhat = A_ee - 1/4 H_eo A_oo^-1 H_oe,  eta_hat_e = eta_e + 1/2 H_eo A_oo^-1 eta_o,
//   psi_o = A_oo^-1 (eta_o + 1/2 H_oe psi_e).
//
// CG_EO     : CG on Dhat^+ Dhat psi_e = Dhat^+ eta_hat_e (tracking s = eta_hat - Dhat psi_e), all FP64,
//             the plain FP64 even-odd CG baseline.  Judged by the full FP64 true residual.
// MP_CGNR   : FP64 outer defect correction around an inner full-lattice CGNR on D M in FP32 (M the
//             learned network or 1), robust where D is indefinite (below).
// MP_CG_EO  : FP64 outer defect correction r = eta - D psi (FP64 D, FP64 norms), around an inner
//             CG whose iteration runs in FP32 vectors with the Dhat applications in inner_prec
//             (FP32, or 16-bit spinors/links/clover with per-site norms), with FP32 reliable
//             updates: when ||s|| has fallen by reliable_delta since the last update, the inner
//             solution is folded into an FP32 accumulator and s is recomputed with the FP32 Dhat.
// Every global inner product and norm is an FP64 reduction.
#include <chrono>
#include <cmath>
#include <cstring>

#include "reduce.cuh"
#include "sap.cuh"

namespace qxd {

enum {
  // FP64
  WS_R64 = 0,   // full residual field [2][12][sv]
  WS_T64,       // full temporary
  WS_BH64,      // even-half vectors [12][sv]
  WS_XE64,
  WS_S64,
  WS_RR64,
  WS_P64,
  WS_Q64,
  WS_TO64,
  // FP32 even/odd halves [6][sv] float4
  WS_BH32,
  WS_Y32,
  WS_X32,
  WS_S32,
  WS_RR32,
  WS_P32,
  WS_Q32,
  WS_TO32,
  // 16-bit halves [6][sv] uint2 and their norms [sv]
  WS_P16,
  WS_S16,
  WS_TO16,
  WS_NRM16,     // 3 norm arrays
  WS_NRM16B,    // 2 norm arrays for full-field 16-bit applies
  WS_R32,       // FP32 copy of the full outer residual
  WS_TO32B,     // FP32 odd-half temporary of the outer correction
  // slots 24..27 belong to the API; BiCGStab's extra vectors reuse the CG ones (RR32 = r_hat,
  // Q32 = v, TO32 = t, S32 = s, X32 = x, P32 = p) plus this one:
  WS_R32B = 28, // BiCGStab residual r
  WS_XB64 = 45, // FP64 copy of x, kept while a failed inner round's progress is tried
};

#define TRY(x)                      \
  do {                              \
    qxd_status _s = (x);            \
    if (_s != QXD_OK) return _s;    \
  } while (0)

template <typename T>
static qxd_status get(qxd_lattice* lat, int slot, size_t bytes, T** out) {
  void* p;
  qxd_status st = ensure_work(lat, slot, bytes, &p);
  *out = (T*)p;
  return st;
}

qxd_status apply_D64(qxd_lattice* lat, const double2* in, double2* out) {
  const i64 h = 12 * lat->sv;
  TRY(hop64(lat, 0, EPI_DFULL, 0, in + h, in, out, 0.0));
  TRY(hop64(lat, 1, EPI_DFULL, 0, in, in + h, out + h, 0.0));
  return QXD_OK;
}

// out_e = Dhat in_e (dag: gamma5 Dhat gamma5), FP64, tmp_o odd-half scratch
static qxd_status dhat64(qxd_lattice* lat, const double2* in, double2* out, double2* tmp, int dag) {
  TRY(hop64(lat, 1, EPI_INV, dag, in, nullptr, tmp, 1.0));
  TRY(hop64(lat, 0, EPI_DHAT2, dag, tmp, in, out, -0.25));
  return QXD_OK;
}

static qxd_status dhat32(qxd_lattice* lat, const float4* in, float4* out, float4* tmp, int dag) {
  TRY(hop32(lat, 1, EPI_INV, dag, in, nullptr, tmp, 1.0f));
  TRY(hop32(lat, 0, EPI_DHAT2, dag, tmp, in, out, -0.25f));
  return QXD_OK;
}

// 16-bit operator: in16 (with norm) -> out FP32
static qxd_status dhat16(qxd_lattice* lat, int bf16, const uint2* in, const float* in_n, float4* out, uint2* tmp,
                         float* tmp_n, int dag) {
  TRY(hop16(lat, bf16, 1, EPI_INV, dag, in, in_n, nullptr, nullptr, tmp, tmp_n, nullptr, 1.0f));
  TRY(hop16(lat, bf16, 0, EPI_DHAT2, dag, tmp, tmp_n, in, in_n, nullptr, nullptr, out, -0.25f));
  return QXD_OK;
}

qxd_status apply_dhat_prec(qxd_lattice* lat, int prec, const double2* in64, double2* out64, int dag) {
  const i64 sv = lat->sv;
  if (prec == QXD_F64) {
    double2* t;
    TRY(get(lat, WS_TO64, sizeof(double2) * 12 * sv, &t));
    return dhat64(lat, in64, out64, t, dag);
  }
  float4 *a, *b, *t;
  TRY(get(lat, WS_P32, sizeof(float4) * 6 * sv, &a));
  TRY(get(lat, WS_Q32, sizeof(float4) * 6 * sv, &b));
  TRY(get(lat, WS_TO32, sizeof(float4) * 6 * sv, &t));
  TRY(f64_to_f32(lat, in64, a, 6 * sv));
  if (prec == QXD_F32) {
    TRY(dhat32(lat, a, b, t, dag));
  } else {
    int bf = prec == QXD_BF16N;
    uint2 *a16, *t16;
    float* nrm;
    TRY(get(lat, WS_P16, sizeof(uint2) * 6 * sv, &a16));
    TRY(get(lat, WS_TO16, sizeof(uint2) * 6 * sv, &t16));
    TRY(get(lat, WS_NRM16, sizeof(float) * 3 * sv, &nrm));
    TRY(f32_to_n16(lat, a, a16, nrm, bf));
    TRY(dhat16(lat, bf, a16, nrm, b, t16, nrm + sv, dag));
  }
  TRY(f32_to_f64(lat, b, out64, 6 * sv));
  return QXD_OK;
}

// full D in a lower precision (both parities), FP64 in/out
qxd_status apply_D_prec(qxd_lattice* lat, int prec, const double2* in64, double2* out64) {
  const i64 sv = lat->sv;
  if (prec == QXD_F64) return apply_D64(lat, in64, out64);
  float4 *a, *b;
  TRY(get(lat, WS_BH32, sizeof(float4) * 12 * sv, &a));  // full field (two halves)
  TRY(get(lat, WS_Y32, sizeof(float4) * 12 * sv, &b));
  TRY(f64_to_f32(lat, in64, a, 12 * sv));
  if (prec == QXD_F32) {
    TRY(hop32(lat, 0, EPI_DFULL, 0, a + 6 * sv, a, b, 0.f));
    TRY(hop32(lat, 1, EPI_DFULL, 0, a, a + 6 * sv, b + 6 * sv, 0.f));
  } else {
    int bf = prec == QXD_BF16N;
    uint2* a16;
    float* nrm;
    TRY(get(lat, WS_S16, sizeof(uint2) * 12 * sv, &a16));
    TRY(get(lat, WS_NRM16B, sizeof(float) * 2 * sv, &nrm));
    TRY(f32_to_n16(lat, a, a16, nrm, bf));
    TRY(f32_to_n16(lat, a + 6 * sv, a16 + 6 * sv, nrm + sv, bf));
    TRY(hop16(lat, bf, 0, EPI_DFULL, 0, a16 + 6 * sv, nrm + sv, a16, nrm, nullptr, nullptr, b, 0.f));
    TRY(hop16(lat, bf, 1, EPI_DFULL, 0, a16, nrm, a16 + 6 * sv, nrm + sv, nullptr, nullptr, b + 6 * sv, 0.f));
  }
  TRY(f32_to_f64(lat, b, out64, 12 * sv));
  return QXD_OK;
}

// ------------------------------------------------------------------------------------------
// FP64 CGLS on Dhat: solve Dhat xe = bh to ||bh - Dhat xe|| <= target (absolute)
// ------------------------------------------------------------------------------------------
static qxd_status cgls64(qxd_lattice* lat, const double2* bh, double2* xe, double target, int maxiter,
                         int check_every, int* iters) {
  const i64 sv = lat->sv, n = 12 * sv;
  const size_t hb = sizeof(double2) * n;
  double2 *s, *rr, *p, *q, *t;
  TRY(get(lat, WS_S64, hb, &s));
  TRY(get(lat, WS_RR64, hb, &rr));
  TRY(get(lat, WS_P64, hb, &p));
  TRY(get(lat, WS_Q64, hb, &q));
  TRY(get(lat, WS_TO64, hb, &t));
  TRY(blas_zero(lat, xe, hb));
  TRY(blas_copy(lat, s, bh, hb));
  TRY(dhat64(lat, s, rr, t, 1));
  TRY(blas_copy(lat, p, rr, hb));
  TRY(blas_norm2_64(lat, rr, n, SC_GAMMA));
  int it = 0;
  double ss;
  TRY(blas_norm2_64(lat, s, n, SC_SS));
  TRY(read_scalars(lat, SC_SS, 1, &ss));
  while (std::sqrt(ss) > target && it < maxiter) {
    TRY(dhat64(lat, p, q, t, 0));
    TRY(blas_norm2_64(lat, q, n, SC_QQ));
    TRY(cg_update_xs_64(lat, xe, p, s, q, n));
    TRY(dhat64(lat, s, rr, t, 1));
    TRY(blas_norm2_64(lat, rr, n, SC_GAMMA_NEW));
    TRY(cg_update_p_64(lat, rr, p, n));
    ++it;
    if (it % check_every == 0) {
      TRY(read_scalars(lat, SC_SS, 1, &ss));
      if (!std::isfinite(ss)) {
        *iters = it;
        return fail(lat, QXD_ENOCONV, "non-finite residual in the FP64 CG");
      }
    }
  }
  *iters = it;
  return QXD_OK;
}

// ------------------------------------------------------------------------------------------
// Inner mixed-precision CGLS: FP32 vectors, Dhat in `prec`, FP32 reliable updates.
// Solves Dhat y = bh32 to ||bh32 - Dhat y|| <= target; y accumulates into y32.
// ------------------------------------------------------------------------------------------
static qxd_status inner_mp(qxd_lattice* lat, int prec, const float4* bh, float4* y, double target, double delta,
                           int maxiter, int check_every, int* iters, int* nrel) {
  const i64 sv = lat->sv, n4 = 6 * sv;
  const size_t hb = sizeof(float4) * n4;
  float4 *x, *s, *rr, *p, *q, *t;
  TRY(get(lat, WS_X32, hb, &x));
  TRY(get(lat, WS_S32, hb, &s));
  TRY(get(lat, WS_RR32, hb, &rr));
  TRY(get(lat, WS_P32, hb, &p));
  TRY(get(lat, WS_Q32, hb, &q));
  TRY(get(lat, WS_TO32, hb, &t));
  const bool low = prec == QXD_F16N || prec == QXD_BF16N;
  const int bf = prec == QXD_BF16N;
  uint2 *p16 = nullptr, *s16 = nullptr, *t16 = nullptr;
  float* nrm = nullptr;
  if (low) {
    TRY(get(lat, WS_P16, sizeof(uint2) * n4, &p16));
    TRY(get(lat, WS_S16, sizeof(uint2) * n4, &s16));
    TRY(get(lat, WS_TO16, sizeof(uint2) * n4, &t16));
    TRY(get(lat, WS_NRM16, sizeof(float) * 3 * sv, &nrm));
  }
  float* p16n = nrm;
  float* s16n = nrm ? nrm + sv : nullptr;
  float* t16n = nrm ? nrm + 2 * sv : nullptr;

  // out = Dhat in (dag: Dhat^+), then ||out||^2 into the device scalar `slot`
  auto apply = [&](const float4* in32, const uint2* in16, const float* in16n, float4* out, int dag,
                   int slot) -> qxd_status {
    if (low)
      TRY(dhat16(lat, bf, in16, in16n, out, t16, t16n, dag));
    else
      TRY(dhat32(lat, in32, out, t, dag));
    return blas_norm2_32(lat, out, n4, slot);
  };

  // s = bh - Dhat y (y is zero on entry, so s = bh); rr = Dhat^+ s; p = rr
  TRY(blas_zero(lat, x, hb));
  TRY(blas_copy(lat, s, bh, hb));
  if (low) TRY(f32_to_n16(lat, s, s16, s16n, bf));
  TRY(apply(s, s16, s16n, rr, 1, SC_GAMMA));
  TRY(blas_copy(lat, p, rr, hb));
  if (low) TRY(f32_to_n16(lat, p, p16, p16n, bf));
  TRY(blas_norm2_32(lat, s, n4, SC_SS));
  double ss;
  TRY(read_scalars(lat, SC_SS, 1, &ss));
  double rmax = std::sqrt(ss);
  int it = 0, rel = 0;
  while (std::sqrt(ss) > target && it < maxiter) {
    // q = Dhat p, ||q||^2; x += alpha p, s -= alpha q (+ 16-bit s); rr = Dhat^+ s, ||rr||^2;
    // p = rr + beta p (+ 16-bit p)
    TRY(apply(p, p16, p16n, q, 0, SC_QQ));
    TRY(cg_update_xs_32(lat, x, p, s, q, low ? s16 : nullptr, s16n, bf));
    TRY(apply(s, s16, s16n, rr, 1, SC_GAMMA_NEW));
    TRY(cg_update_p_32(lat, rr, p, low ? p16 : nullptr, p16n, bf));
    ++it;
    if (it % check_every == 0) {
      TRY(read_scalars(lat, SC_SS, 1, &ss));
      if (!std::isfinite(ss)) {  // y keeps what the reliable updates folded in; x is dropped
        *iters = it;
        *nrel = rel;
        return fail(lat, QXD_ENOCONV, "non-finite residual in the inner CG");
      }
      double sn = std::sqrt(ss);
      if (sn > rmax) rmax = sn;
      if (sn < delta * rmax || sn <= target) {
        // reliable update: fold x into y, recompute s = bh - Dhat32 y in FP32
        TRY(blas_axpy_32(lat, 1.0f, x, y, n4));
        TRY(blas_zero(lat, x, hb));
        TRY(dhat32(lat, y, q, t, 0));
        TRY(blas_copy(lat, s, bh, hb));
        TRY(blas_axpy_32(lat, -1.0f, q, s, n4));
        TRY(blas_norm2_32(lat, s, n4, SC_SS));
        TRY(read_scalars(lat, SC_SS, 1, &ss));
        if (!std::isfinite(ss)) {  // a non-finite update reached y itself
          *iters = it;
          *nrel = rel;
          return fail(lat, QXD_ENOCONV, "non-finite residual in the inner CG");
        }
        rmax = std::sqrt(ss);
        ++rel;
        if (std::sqrt(ss) > target) {
          // keep p; refresh rr and gamma from the new residual
          if (low) TRY(f32_to_n16(lat, s, s16, s16n, bf));
          TRY(apply(s, s16, s16n, rr, 1, SC_GAMMA));
        }
      }
    }
  }
  // fold the rest
  TRY(blas_axpy_32(lat, 1.0f, x, y, n4));
  *iters = it;
  *nrel = rel;
  return QXD_OK;
}

// ------------------------------------------------------------------------------------------
// Inner mixed-precision BiCGStab on Dhat: FP32 vectors, Dhat in `prec`, FP32 reliable updates
// (each one recomputes r = bh - Dhat32 y and restarts with r_hat = p = r).
// ------------------------------------------------------------------------------------------
static qxd_status inner_bicg(qxd_lattice* lat, int prec, const float4* bh, float4* y, double target, double delta,
                             int maxiter, int check_every, int* iters, int* nrel) {
  const i64 sv = lat->sv, n4 = 6 * sv;
  const size_t hb = sizeof(float4) * n4;
  float4 *x, *r, *rh, *p, *v, *s, *t, *tmp;
  TRY(get(lat, WS_X32, hb, &x));
  TRY(get(lat, WS_R32B, hb, &r));
  TRY(get(lat, WS_RR32, hb, &rh));
  TRY(get(lat, WS_P32, hb, &p));
  TRY(get(lat, WS_Q32, hb, &v));
  TRY(get(lat, WS_S32, hb, &s));
  TRY(get(lat, WS_TO32, hb, &t));
  TRY(get(lat, WS_BH32 + 0, sizeof(float4) * 12 * sv, &tmp));  // only its odd half is used below
  float4* tmp_o = tmp + 6 * sv;
  const bool low = prec == QXD_F16N || prec == QXD_BF16N;
  const int bf = prec == QXD_BF16N;
  uint2 *p16 = nullptr, *s16 = nullptr, *t16 = nullptr;
  float* nrm = nullptr;
  if (low) {
    TRY(get(lat, WS_P16, sizeof(uint2) * n4, &p16));
    TRY(get(lat, WS_S16, sizeof(uint2) * n4, &s16));
    TRY(get(lat, WS_TO16, sizeof(uint2) * n4, &t16));
    TRY(get(lat, WS_NRM16, sizeof(float) * 3 * sv, &nrm));
  }
  float* p16n = nrm;
  float* s16n = nrm ? nrm + sv : nullptr;
  float* t16n = nrm ? nrm + 2 * sv : nullptr;
  auto apply = [&](const float4* in32, const uint2* in16, const float* in16n, float4* out) -> qxd_status {
    if (low) return dhat16(lat, bf, in16, in16n, out, t16, t16n, 0);
    return dhat32(lat, in32, out, tmp_o, 0);
  };
  // restart from the current residual r: r_hat = p = r, rho = <r, r>
  auto restart = [&]() -> qxd_status {
    TRY(blas_copy(lat, rh, r, hb));
    TRY(bicg_copy(lat, r, p, low ? p16 : nullptr, p16n, bf));
    TRY(bicg_cdot(lat, rh, r, SC_RHO));
    return QXD_OK;
  };
  TRY(set_scalar(lat, SC_ACTIVE, 1.0));
  TRY(blas_zero(lat, x, hb));
  TRY(blas_copy(lat, r, bh, hb));
  TRY(restart());
  TRY(blas_norm2_32(lat, r, n4, SC_RN));
  double rn2;
  TRY(read_scalars(lat, SC_RN, 1, &rn2));
  double rmax = std::sqrt(rn2);
  int it = 0, rel = 0, breakdowns = 0;
  while (std::sqrt(rn2) > target && it < maxiter) {
    TRY(apply(p, p16, p16n, v));                                  // v = Dhat p
    TRY(bicg_cdot(lat, rh, v, SC_RV));                            // <r_hat, v>
    TRY(bicg_s(lat, r, v, s, low ? s16 : nullptr, s16n, bf));     // s = r - alpha v
    TRY(apply(s, s16, s16n, t));                                  // t = Dhat s
    TRY(bicg_ts(lat, t, s));                                      // <t, s>, <t, t>
    TRY(bicg_xr(lat, x, p, s, t, rh, r));                         // x, r, <r_hat, r>, ||r||^2
    TRY(bicg_p(lat, r, v, p, low ? p16 : nullptr, p16n, bf));     // p, rho
    ++it;
    if (it % check_every == 0) {
      TRY(read_scalars(lat, SC_RN, 1, &rn2));
      const bool broke = !std::isfinite(rn2);  // breakdown (e.g. <r_hat, v> = 0): drop x, restart
      if (broke && ++breakdowns > 10) {  // y keeps what the reliable updates folded in
        *iters = it;
        *nrel = rel;
        return fail(lat, QXD_ENOCONV, "repeated breakdown in the inner BiCGStab");
      }
      double rn = broke ? 0.0 : std::sqrt(rn2);
      if (rn > rmax) rmax = rn;
      if (broke || rn < delta * rmax || rn <= target) {
        if (!broke) TRY(blas_axpy_32(lat, 1.0f, x, y, n4));
        TRY(blas_zero(lat, x, hb));
        TRY(dhat32(lat, y, v, tmp_o, 0));
        TRY(blas_copy(lat, r, bh, hb));
        TRY(blas_axpy_32(lat, -1.0f, v, r, n4));
        TRY(blas_norm2_32(lat, r, n4, SC_RN));
        TRY(read_scalars(lat, SC_RN, 1, &rn2));
        if (!std::isfinite(rn2)) {  // a non-finite update reached y itself
          *iters = it;
          *nrel = rel;
          return fail(lat, QXD_ENOCONV, "non-finite residual in the inner BiCGStab");
        }
        rmax = std::sqrt(rn2);
        ++rel;
        if (std::sqrt(rn2) > target) TRY(restart());
      }
    }
  }
  TRY(blas_axpy_32(lat, 1.0f, x, y, n4));
  *iters = it;
  *nrel = rel;
  return QXD_OK;
}

// ------------------------------------------------------------------------------------------
// Inner CGNR on the full lattice, FP32, right-preconditioned by the network M (or M = 1):
// CG on (D M)^+ (D M) y = (D M)^+ rhs, accumulating the correction e = M y directly (e += alpha
// M p, since M is linear), s = rhs - D e tracked, FP32 reliable updates recompute s = rhs - D e
// when ||s|| has fallen by delta and restart the CG there.  The normal equations are Hermitian positive definite whatever
// the spectrum of D, so the iteration converges where GCR and BiCGStab stagnate on an indefinite
// D; M^+ is the adjoint network and D^+ = gamma5 D gamma5.
// ------------------------------------------------------------------------------------------
enum { WS_NR_S = 52, WS_NR_Z, WS_NR_P, WS_NR_W, WS_NR_Q, WS_NR_T };

static qxd_status cgnr32(qxd_lattice* lat, qxd_net* net, const float4* rhs, float4* e, double target, double delta,
                         int maxiter, int check_every, int* iters, int* nrel) {
  const i64 sv = lat->sv, n4 = 12 * sv;
  const size_t fb = sizeof(float4) * n4;
  float4 *s, *z, *p, *w, *q, *t;
  TRY(get(lat, WS_NR_S, fb, &s));
  TRY(get(lat, WS_NR_Z, fb, &z));
  TRY(get(lat, WS_NR_P, fb, &p));
  TRY(get(lat, WS_NR_W, fb, &w));
  TRY(get(lat, WS_NR_Q, fb, &q));
  TRY(get(lat, WS_NR_T, fb, &t));
  // out = D in (dag: D^+ = gamma5 D gamma5), full FP32 fields
  auto dfull = [&](const float4* in, float4* out, int dag) -> qxd_status {
    TRY(hop32(lat, 0, EPI_DFULL, dag, in + 6 * sv, in, out, 0.f));
    return hop32(lat, 1, EPI_DFULL, dag, in, in + 6 * sv, out + 6 * sv, 0.f);
  };
  // out = M^+ D^+ in
  auto normal_rhs = [&](const float4* in, float4* out) -> qxd_status {
    if (!net) return dfull(in, out, 1);
    TRY(dfull(in, t, 1));
    return net_apply_adj32(net, t, out);
  };
  TRY(blas_copy(lat, s, rhs, fb));
  TRY(blas_zero(lat, e, fb));
  TRY(normal_rhs(s, z));
  TRY(blas_copy(lat, p, z, fb));
  TRY(blas_norm2_32(lat, z, n4, SC_GAMMA));
  TRY(blas_norm2_32(lat, s, n4, SC_SS));
  double ss;
  TRY(read_scalars(lat, SC_SS, 1, &ss));
  double rmax = std::sqrt(ss);
  int it = 0, rel = 0;
  while (std::sqrt(ss) > target && it < maxiter) {
    const float4* wp = p;
    if (net) {
      TRY(net_apply32(net, p, w));  // w = M p
      wp = w;
    }
    TRY(dfull(wp, q, 0));                                     // q = D M p
    TRY(blas_norm2_32(lat, q, n4, SC_QQ));
    TRY(cg_update_xs_32_full(lat, e, wp, s, q));              // e += alpha M p, s -= alpha q, ||s||^2
    TRY(normal_rhs(s, z));                                    // z = M^+ D^+ s
    TRY(blas_norm2_32(lat, z, n4, SC_GAMMA_NEW));
    TRY(cg_update_p_32_full(lat, z, p));                      // p = z + beta p
    ++it;
    if (it % check_every == 0) {
      TRY(read_scalars(lat, SC_SS, 1, &ss));
      if (!std::isfinite(ss)) {  // e keeps what it had before this check
        *iters = it;
        *nrel = rel;
        return fail(lat, QXD_ENOCONV, "non-finite residual in the inner CGNR");
      }
      const double sn = std::sqrt(ss);
      if (sn > rmax) rmax = sn;
      if (sn < delta * rmax || sn <= target) {
        // reliable update: s = rhs - D e in FP32, then restart from it (p = z).  Keeping the old
        // p here lets FP32 rounding steer it into near-null directions of D on ill-conditioned
        // fields, where the iteration then diverges (measured: 16^3x32 at m0 = -0.12).
        TRY(dfull(e, q, 0));
        TRY(blas_copy(lat, s, rhs, fb));
        TRY(blas_axpy_32(lat, -1.0f, q, s, n4));
        TRY(blas_norm2_32(lat, s, n4, SC_SS));
        TRY(read_scalars(lat, SC_SS, 1, &ss));
        if (!std::isfinite(ss)) {  // a non-finite update reached e itself
          *iters = it;
          *nrel = rel;
          return fail(lat, QXD_ENOCONV, "non-finite residual in the inner CGNR");
        }
        rmax = std::sqrt(ss);
        ++rel;
        if (std::sqrt(ss) > target) {
          TRY(normal_rhs(s, z));
          TRY(blas_copy(lat, p, z, fb));
          TRY(blas_norm2_32(lat, z, n4, SC_GAMMA));
        }
      }
    }
  }
  *iters = it;
  *nrel = rel;
  if (net) TRY(net_check(net));
  return QXD_OK;
}

// The inner flexible GCR of QXD_SOLVER_MP_FGCR_NET lives in fgcr.cu (device-resident coefficients).
qxd_status fgcr32(qxd_lattice* lat, qxd_net* net, const SapSpec* sap, int m, int reorth, const float4* rhs, float4* y,
                  double target, int maxiter, int check_every, int* iters);

static qxd_status solve_impl(qxd_lattice* lat, double2* x, const double2* b, const qxd_solve_params* prm,
                             qxd_solve_info* info);

// A failed solve leaves x usable as a starting point when its true residual is finite and below
// that of x = 0.  solve_impl reports NaN until it has computed the residual of the x it returns,
// so a residual that was never computed is never trusted.
static bool usable_iterate(const qxd_solve_info& i) { return std::isfinite(i.true_rel_res) && i.true_rel_res < 1.0; }

// Recovery chain after a missed tolerance (stagnation, breakdown, an expired wait): first the
// FP32-inner restart of a 16-bit MP solve (restart_f32), then the plain fallback solver
// (fallback).  Argument errors and CUDA failures are returned as they are.
qxd_status solve(qxd_lattice* lat, double2* x, const double2* b, const qxd_solve_params* prm, qxd_solve_info* info) {
  auto t0 = std::chrono::steady_clock::now();
  qxd_solve_info own;
  qxd_solve_info* inf = info ? info : &own;  // solve_impl fills every field
  qxd_status st = solve_impl(lat, x, b, prm, inf);
  if (st != QXD_OK && inf->status == QXD_OK) inf->status = st;  // early failure: record it
  auto recoverable = [](qxd_status s) { return s == QXD_ENOCONV || s == QXD_ETIMEOUT; };
  const bool mp16 = (prm->solver == QXD_SOLVER_MP_CG_EO || prm->solver == QXD_SOLVER_MP_BICGSTAB_EO) &&
                    (prm->inner_prec == QXD_F16N || prm->inner_prec == QXD_BF16N);
  if (recoverable(st) && prm->restart_f32 && mp16 && prm->maxiter > inf->iters_inner) {
    qxd_solve_params rp = *prm;
    rp.inner_prec = QXD_F32;
    rp.maxiter = prm->maxiter - inf->iters_inner;
    rp.use_x0 = usable_iterate(*inf);
    qxd_solve_info ri;
    std::memset(&ri, 0, sizeof(ri));
    st = solve_impl(lat, x, b, &rp, &ri);
    if (st != QXD_OK && ri.status == QXD_OK) ri.status = st;
    inf->iters_inner += ri.iters_inner;
    inf->iters_outer += ri.iters_outer;
    inf->reliable_updates += ri.reliable_updates;
    inf->true_rel_res = ri.true_rel_res;
    inf->status = ri.status;
    inf->fallback_used |= 2;
  }
  if (recoverable(st) && prm->fallback >= 0) {
    qxd_solve_params fp;
    qxd_default_params(&fp);
    fp.solver = prm->fallback;
    fp.tol = prm->tol;
    fp.on_device = prm->on_device;
    fp.check_every = prm->check_every;
    fp.use_x0 = usable_iterate(*inf);
    qxd_solve_info fi;
    std::memset(&fi, 0, sizeof(fi));
    st = solve_impl(lat, x, b, &fp, &fi);
    if (st != QXD_OK && fi.status == QXD_OK) fi.status = st;
    fi.fallback_used = inf->fallback_used | 1;
    *inf = fi;
  }
  inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

static qxd_status solve_impl(qxd_lattice* lat, double2* x, const double2* b, const qxd_solve_params* prm,
                             qxd_solve_info* info) {
  auto t0 = std::chrono::steady_clock::now();
  if (info) {
    // until a residual is computed for x, none is reported: an early error leaves NaN, which the
    // recovery chain reads as "x unusable"
    std::memset(info, 0, sizeof(*info));
    info->true_rel_res = std::nan("");
    info->status = QXD_ENOCONV;
  }
  const i64 sv = lat->sv, nh = 12 * sv, nf = 24 * sv;
  const size_t fb = sizeof(double2) * nf, hb = sizeof(double2) * nh;
  double2 *r, *tf, *bh, *xe, *to;
  TRY(get(lat, WS_R64, fb, &r));
  TRY(get(lat, WS_T64, fb, &tf));
  TRY(get(lat, WS_BH64, hb, &bh));
  TRY(get(lat, WS_XE64, hb, &xe));
  TRY(get(lat, WS_TO64, hb, &to));
  const bool mp = prm->solver == QXD_SOLVER_MP_CG_EO || prm->solver == QXD_SOLVER_MP_BICGSTAB_EO;
  const bool gcr = prm->solver == QXD_SOLVER_MP_FGCR_NET || prm->solver == QXD_SOLVER_MP_SAP_GCR ||
                   prm->solver == QXD_SOLVER_MP_DFL_SAP_GCR || prm->solver == QXD_SOLVER_MP_MG_GCR;
  const bool cgnr = prm->solver == QXD_SOLVER_MP_CGNR;
  float4 *bh32 = nullptr, *y32 = nullptr, *r32 = nullptr, *to32 = nullptr;
  if (mp) {
    TRY(get(lat, WS_BH32, sizeof(float4) * 12 * sv, &bh32));  // sized for full fields (apply_D_prec shares it)
    TRY(get(lat, WS_Y32, sizeof(float4) * 12 * sv, &y32));
    TRY(get(lat, WS_R32, sizeof(float4) * 12 * sv, &r32));
    TRY(get(lat, WS_TO32B, sizeof(float4) * 6 * sv, &to32));
  }
  double bn2;
  TRY(blas_norm2_64(lat, b, nf, SC_TMP0));
  TRY(read_scalars(lat, SC_TMP0, 1, &bn2));
  const double bnorm = std::sqrt(bn2);
  // with an initial guess the first round starts from r = b - D x (b = 0 has the solution 0)
  const bool from_x0 = prm->use_x0 != 0 && bnorm != 0.0;
  if (!from_x0) TRY(blas_zero(lat, x, fb));
  int total = 0, outer = 0, nrel_total = 0;
  double rel = 1.0;
  qxd_status result = QXD_ENOCONV;
  const char* why = "tolerance not reached within maxiter / max_outer";
  if (bnorm == 0.0) {
    rel = 0.0;
    result = QXD_OK;
  }
  auto fill_info = [&](double res, int status) {
    if (!info) return;
    info->iters_inner = total;
    info->iters_outer = outer;
    info->reliable_updates = nrel_total;
    info->true_rel_res = res;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->status = status;
  };
  // r = b - D x and its relative norm (FP64)
  auto true_residual = [&](double* out_rel) -> qxd_status {
    TRY(apply_D64(lat, x, tf));
    TRY(blas_copy(lat, r, b, fb));
    TRY(blas_axpy_64(lat, -1.0, 0.0, tf, r, nf));
    double rn2;
    TRY(blas_norm2_64(lat, r, nf, SC_TMP0));
    TRY(read_scalars(lat, SC_TMP0, 1, &rn2));
    *out_rel = std::sqrt(rn2) / bnorm;
    return QXD_OK;
  };
  const int max_outer = prm->max_outer > 0 ? prm->max_outer : 20;
  for (; result != QXD_OK && outer <= max_outer; ++outer) {
    if (outer == 0 && !from_x0) {
      TRY(blas_copy(lat, r, b, fb));
      rel = 1.0;
    } else {
      TRY(true_residual(&rel));
    }
    if (!std::isfinite(rel)) {
      fill_info(rel, QXD_ENOCONV);
      return fail(lat, QXD_ENOCONV, "non-finite residual");
    }
    if (rel <= prm->tol) {
      result = QXD_OK;
      break;
    }
    if (outer == max_outer || total >= prm->maxiter) break;
    const double rnorm = rel * bnorm;
    int it = 0, nrel = 0;
    // status of the inner solve: QXD_ENOCONV means it gave up early (breakdown, non-finite
    // residual) after `it` iterations; any other failure is returned as it is
    qxd_status ist = QXD_OK;
    auto inner_status = [&](qxd_status s) -> bool { ist = s; return s == QXD_OK || s == QXD_ENOCONV; };
    const double target = 0.5 * prm->tol * bnorm;
    if (cgnr) {
      // the correction D e = r on the full lattice by CGNR on D M (M the network, or 1), FP32
      float4 *r32f, *e32;
      TRY(get(lat, WS_R32, sizeof(float4) * 12 * sv, &r32f));
      TRY(get(lat, WS_BH32, sizeof(float4) * 12 * sv, &e32));
      TRY(f64_to_f32(lat, r, r32f, 12 * sv));
      double inner_target = prm->inner_tol * rnorm;
      if (inner_target < target) inner_target = target;
      if (!inner_status(cgnr32(lat, const_cast<qxd_net*>(prm->net), r32f, e32, inner_target, prm->reliable_delta,
                               prm->maxiter - total, prm->check_every > 0 ? prm->check_every : 1, &it, &nrel)))
        return ist;
      if (ist != QXD_OK) TRY(blas_copy(lat, tf, x, fb));
      TRY(blas_acc_f32_into_f64(lat, e32, x, 12 * sv));
    } else if (gcr) {
      // the correction D e = r on the full lattice by FGCR with the network or SAP, FP32
      float4 *r32f, *e32;
      TRY(get(lat, WS_R32, sizeof(float4) * 12 * sv, &r32f));
      TRY(get(lat, WS_BH32, sizeof(float4) * 12 * sv, &e32));
      TRY(f64_to_f32(lat, r, r32f, 12 * sv));
      TRY(blas_zero(lat, e32, sizeof(float4) * 12 * sv));
      double inner_target = prm->inner_tol * rnorm;
      if (inner_target < target) inner_target = target;
      SapSpec sp;
      const bool with_sap = prm->solver == QXD_SOLVER_MP_SAP_GCR || prm->solver == QXD_SOLVER_MP_DFL_SAP_GCR ||
                            prm->solver == QXD_SOLVER_MP_MG_GCR;
      if (with_sap) {
        for (int mu = 0; mu < 4; ++mu) sp.block[mu] = prm->sap_block[mu];
        sp.ncy = prm->sap_ncy;
        sp.nmr = prm->sap_nmr;
        sp.dfl = prm->solver == QXD_SOLVER_MP_DFL_SAP_GCR;
        sp.mg = prm->solver == QXD_SOLVER_MP_MG_GCR;
      }
      if (!inner_status(fgcr32(lat, with_sap ? nullptr : const_cast<qxd_net*>(prm->net), with_sap ? &sp : nullptr,
                               prm->gcr_restart, prm->gcr_reorth, r32f, e32, inner_target, prm->maxiter - total,
                               prm->check_every, &it)))
        return ist;
      if (ist != QXD_OK) TRY(blas_copy(lat, tf, x, fb));
      TRY(blas_acc_f32_into_f64(lat, e32, x, 12 * sv));
    } else if (!mp) {
      // Schur source bh = r_e + 1/2 H_eo A_oo^-1 r_o, CG, reconstruct x_o += A_oo^-1 (r_o + 1/2 H_oe xe)
      TRY(clover_apply64(lat, 1, 1, r + nh, to));
      TRY(hop64(lat, 0, EPI_XPAY, 0, to, r, bh, 0.5));
      if (!inner_status(cgls64(lat, bh, xe, target, prm->maxiter - total,
                               prm->check_every > 0 ? prm->check_every : 1, &it)))
        return ist;
      if (ist != QXD_OK) TRY(blas_copy(lat, tf, x, fb));
      TRY(hop64(lat, 1, EPI_INVXPAY, 0, xe, r + nh, to, 0.5));
      TRY(blas_axpy_64(lat, 1.0, 0.0, xe, x, nh));
      TRY(blas_axpy_64(lat, 1.0, 0.0, to, x + nh, nh));
    } else {
      // the correction equation D e = r only needs the inner accuracy, so its Schur source and
      // reconstruction run in FP32; x accumulates in FP64
      TRY(f64_to_f32(lat, r, r32, 12 * sv));
      TRY(clover_apply32(lat, 1, 1, r32 + 6 * sv, to32));
      TRY(hop32(lat, 0, EPI_XPAY, 0, to32, r32, bh32, 0.5f));
      TRY(blas_zero(lat, y32, sizeof(float4) * 6 * sv));
      double inner_target = prm->inner_tol * rnorm;
      if (inner_target < target) inner_target = target;
      const int every = prm->check_every > 0 ? prm->check_every : 1;
      const bool ok =
          prm->solver == QXD_SOLVER_MP_BICGSTAB_EO
              ? inner_status(inner_bicg(lat, prm->inner_prec, bh32, y32, inner_target, prm->reliable_delta,
                                        prm->maxiter - total, every, &it, &nrel))
              : inner_status(inner_mp(lat, prm->inner_prec, bh32, y32, inner_target, prm->reliable_delta,
                                      prm->maxiter - total, every, &it, &nrel));
      if (!ok) return ist;
      if (ist != QXD_OK) TRY(blas_copy(lat, tf, x, fb));
      TRY(hop32(lat, 1, EPI_INVXPAY, 0, y32, r32 + 6 * sv, to32, 0.5f));
      TRY(blas_acc_f32_into_f64(lat, y32, x, 6 * sv));
      TRY(blas_acc_f32_into_f64(lat, to32, x + nh, 6 * sv));
    }
    total += it;
    nrel_total += nrel;
    if (ist != QXD_OK) {
      // The inner solve gave up early.  Keep what it folded in if that lowers the true
      // residual, else return to the x of this round (saved in tf, copied to XB64 first since
      // the residual below overwrites tf); either way true_rel_res is that of the x returned.
      double2* xb;
      TRY(get(lat, WS_XB64, fb, &xb));
      TRY(blas_copy(lat, xb, tf, fb));
      double rel_new;
      TRY(true_residual(&rel_new));
      if (std::isfinite(rel_new) && rel_new < rel) {
        rel = rel_new;
      } else {
        TRY(blas_copy(lat, x, xb, fb));
      }
      why = "the inner solver gave up (breakdown or non-finite residual)";
      ++outer;
      break;
    }
  }
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  fill_info(rel, result);
  if (result != QXD_OK) return fail(lat, QXD_ENOCONV, why);
  return QXD_OK;
}

}  // namespace qxd
