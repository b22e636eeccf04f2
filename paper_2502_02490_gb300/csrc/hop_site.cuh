// The hop at one output site with its fused epilogue, shared by the hop kernels and the batched
// persistent solver.  (H psi)(x) = sum_mu [(1 - gamma_mu) W_mu(x) psi(x+mu)
//                                       + (1 + gamma_mu) W_mu(x-mu)^dag psi(x-mu)]
// Epilogues: HOP: out = coef H in;  DFULL: out = A same - 1/2 g5? H g5? in (with g5: the parity block
//            of D^+ = gamma5 D gamma5, since A commutes with gamma5);  INV: out = A^-1 (coef H g5? in);
//            DHAT2: out = A same + coef g5? H in;  XPAY: out = same + coef H in;
//            INVXPAY: out = A^-1 (same + coef H in).
#pragma once

#include "hop_common.cuh"

namespace qxd {

// One of the eight hops ("legs": 2*mu + 0 forward, 2*mu + 1 backward) of the software-pipelined
// kernel: decode the raw neighbour spinor and link fetched PF legs earlier, refill the slot with
// the raw data of leg LEG + PF, then project, scale (per-site norm and time-boundary sign, applied
// once to the 6-component half spinor), transport and accumulate.
#ifndef QXD_HOP16_MINB
#define QXD_HOP16_MINB 5  // min resident blocks per SM for the 16-bit kernels (swept 1,4..7 on GB300; 5 best)
#endif

#ifndef QXD_HOP_PF16
#define QXD_HOP_PF16 4  // prefetch depth of the 16-bit kernels (legs in flight); 4 measured best on GB300
#endif

template <int LEG, int PF, typename R, class SIN, class LNK, bool G5IN>
__device__ __forceinline__ void leg_step(const Geom& g, int par, uint32_t cb, const uint32_t nb[8], bool cr_f,
                                         bool cr_b, const SIN& in, const LNK& lk, typename SIN::Raw* sr,
                                         typename LNK::Raw* lr, cplx<R> acc[12]) {
  constexpr int MU = LEG >> 1;
  constexpr bool FWD = (LEG & 1) == 0;
  constexpr int slot = LEG % PF;
  cplx<R> s[12], u[9], h[6], t[6];
  R sc = in.decode(sr[slot], s);
  lk.decode(lr[slot], u);
  if constexpr (LEG + PF < 8) {
    constexpr int nl = LEG + PF;
    sr[slot] = in.fetch(nb[nl]);
    lr[slot] = lk.fetch((nl & 1) ? 1 - par : par, nl >> 1, (nl & 1) ? nb[nl] : cb);
  }
  if (G5IN) {
#pragma unroll
    for (int k = 6; k < 12; ++k) s[k] = neg(s[k]);
  }
  project<R, MU, FWD>(s, h);
  if (MU == 0 && (FWD ? cr_f : cr_b) && g.anti) sc = -sc;
#pragma unroll
  for (int k = 0; k < 6; ++k) h[k] = sc * h[k];
  link_mul<R, !FWD>(u, h, t);
  accumulate<R, MU, FWD>(acc, t);
}

// Epilogue prefetch: for the 16-bit kernels the clover block pair and the diagonal input spinor
// are fetched two legs before the end, so their latency overlaps the last two hops.
template <class T>
struct is16 {
  static constexpr bool value = false;
};
template <class F>
struct is16<Clover16<F>> {
  static constexpr bool value = true;
};

template <typename R, class CLV>
__device__ __forceinline__ void clover_mul_raw(const CLV& cl, const typename CLV::Raw& raw, const cplx<R> v[12],
                                               cplx<R> y[12]) {
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    R r[36];
    cl.decode(raw, blk, r);
    herm6_apply<R>(r, v + 6 * blk, y + 6 * blk);
  }
}

template <typename R, class CLV>
__device__ __forceinline__ void clover_mul(const CLV& cl, int par, i64 cb, const cplx<R> v[12], cplx<R> y[12]) {
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    R r[36];
    cl.load(par, blk, cb, r);
    herm6_apply<R>(r, v + 6 * blk, y + 6 * blk);
  }
}

struct NoSpinor {
  typedef float real;
  template <typename T>
  __device__ __forceinline__ void load(i64, cplx<T>*) const {}
  template <typename T>
  __device__ __forceinline__ void store(i64, const cplx<T>*) const {}
};

template <typename R, class SIN, class SSAME, class SOUT, class LNK, class CLV, int EPI, bool G5, int PF>
__device__ __forceinline__ void hop_site(const Geom& g, int par, uint32_t cb, const SIN& in, const SSAME& same,
                                         const SOUT& out, const LNK& lk, const CLV& cl, R coef,
                                         cplx<R>* keep = nullptr) {  // keep: a copy of the output spinor
  int x[4];
  cb_coords32(g, cb, par, x);
  uint32_t nb[8];
  bool cr_f = false, cr_b = false, c;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    nb[2 * mu] = nbr_cb32(g, x, mu, +1, c);
    if (mu == 0) cr_f = c;
    nb[2 * mu + 1] = nbr_cb32(g, x, mu, -1, c);
    if (mu == 0) cr_b = c;
  }
  typename SIN::Raw sr[PF];
  typename LNK::Raw lr[PF];
#pragma unroll
  for (int l = 0; l < PF; ++l) {
    sr[l] = in.fetch(nb[l]);
    lr[l] = lk.fetch((l & 1) ? 1 - par : par, l >> 1, (l & 1) ? nb[l] : cb);
  }
  cplx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = mk((R)0, (R)0);
  constexpr bool G5IN = G5 && (EPI == EPI_INV || EPI == EPI_DFULL);
  leg_step<0, PF, R, SIN, LNK, G5IN>(g, par, cb, nb, cr_f, cr_b, in, lk, sr, lr, acc);
  leg_step<1, PF, R, SIN, LNK, G5IN>(g, par, cb, nb, cr_f, cr_b, in, lk, sr, lr, acc);
  leg_step<2, PF, R, SIN, LNK, G5IN>(g, par, cb, nb, cr_f, cr_b, in, lk, sr, lr, acc);
  leg_step<3, PF, R, SIN, LNK, G5IN>(g, par, cb, nb, cr_f, cr_b, in, lk, sr, lr, acc);
  leg_step<4, PF, R, SIN, LNK, G5IN>(g, par, cb, nb, cr_f, cr_b, in, lk, sr, lr, acc);
  leg_step<5, PF, R, SIN, LNK, G5IN>(g, par, cb, nb, cr_f, cr_b, in, lk, sr, lr, acc);
  constexpr bool EPF = is16<CLV>::value;  // epilogue prefetch (16-bit kernels)
  constexpr bool USES_CLOVER = EPI != EPI_HOP && EPI != EPI_XPAY;
  constexpr bool USES_SAME = EPI == EPI_DFULL || EPI == EPI_DHAT2 || EPI == EPI_INVXPAY || EPI == EPI_XPAY;
  typename CLV::Raw craw;
  typename SSAME::Raw sraw;
  if constexpr (EPF) {
    if constexpr (USES_CLOVER) craw = cl.fetch(par, cb);
    if constexpr (USES_SAME) sraw = same.fetch(cb);
  }
  leg_step<6, PF, R, SIN, LNK, G5IN>(g, par, cb, nb, cr_f, cr_b, in, lk, sr, lr, acc);
  leg_step<7, PF, R, SIN, LNK, G5IN>(g, par, cb, nb, cr_f, cr_b, in, lk, sr, lr, acc);

  // the diagonal input spinor (prefetched raw data for the 16-bit kernels)
  auto load_same = [&](cplx<R> v[12]) {
    if constexpr (EPF) {
      R n = same.decode(sraw, v);
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = n * v[k];
    } else {
      same.load(cb, v);
    }
  };
  auto cmul = [&](const cplx<R> v[12], cplx<R> y[12]) {
    if constexpr (EPF)
      clover_mul_raw<R, CLV>(cl, craw, v, y);
    else
      clover_mul<R, CLV>(cl, par, cb, v, y);
  };

  cplx<R> o[12];
  if (EPI == EPI_HOP) {
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = coef * acc[k];
  } else if (EPI == EPI_DFULL || EPI == EPI_DHAT2) {
    cplx<R> v[12], y[12];
    load_same(v);
    cmul(v, y);
    R c = EPI == EPI_DFULL ? (R)-0.5 : coef;
    if ((EPI == EPI_DHAT2 || EPI == EPI_DFULL) && G5) {  // DFULL: A same - 1/2 gamma5 H gamma5 in
#pragma unroll
      for (int k = 6; k < 12; ++k) acc[k] = neg(acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = y[k] + c * acc[k];
  } else if (EPI == EPI_INV) {
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = coef * acc[k];
    cmul(acc, o);
  } else if (EPI == EPI_INVXPAY) {
    cplx<R> v[12];
    load_same(v);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = v[k] + coef * acc[k];
    cmul(v, o);
  } else {  // EPI_XPAY
    cplx<R> v[12];
    load_same(v);
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = v[k] + coef * acc[k];
  }
  out.store(cb, o);
  if (keep) {
#pragma unroll
    for (int k = 0; k < 12; ++k) keep[k] = o[k];
  }
}

}  // namespace qxd
