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
// the raw data of leg LEG + PF, then project, transport, and accumulate with the scale (per-site
// norm and time-boundary sign) folded into the accumulation's fused multiply-adds.
#ifndef QXD_HOP16_MINB
#define QXD_HOP16_MINB 5  // min resident blocks per SM for the 16-bit kernels (swept 1,4..7 on GB300; 5 best)
#endif

#ifndef QXD_HOP_PF16
#define QXD_HOP_PF16 4  // prefetch depth of the 16-bit kernels (legs in flight); 4 measured best on GB300
#endif

#ifndef QXD_HOP16_HMATH
#define QXD_HOP16_HMATH 1  // 16-bit hops: spin projection and link product in packed 16-bit arithmetic
#endif

// Packed 16-bit arithmetic of a storage format: one complex number per 32-bit word (re low, im high).
template <class FMT>
struct HM;
template <>
struct HM<H16> {
  typedef __half2 T;
  static __device__ __forceinline__ T word(uint32_t w) {
    T t;
    memcpy(&t, &w, 4);
    return t;
  }
  static __device__ __forceinline__ T two(float a, float b) { return __floats2half2_rn(a, b); }
  static __device__ __forceinline__ T lo2(T a) { return __low2half2(a); }
  static __device__ __forceinline__ T hi2(T a) { return __high2half2(a); }
  static __device__ __forceinline__ cplx<float> f32(T a) {
    const float2 f = __half22float2(a);
    return mk(f.x, f.y);
  }
};
template <>
struct HM<B16> {
  typedef __nv_bfloat162 T;
  static __device__ __forceinline__ T word(uint32_t w) {
    T t;
    memcpy(&t, &w, 4);
    return t;
  }
  static __device__ __forceinline__ T two(float a, float b) { return __floats2bfloat162_rn(a, b); }
  static __device__ __forceinline__ T lo2(T a) { return __low2bfloat162(a); }
  static __device__ __forceinline__ T hi2(T a) { return __high2bfloat162(a); }
  static __device__ __forceinline__ cplx<float> f32(T a) { return mk(__low2float(a), __high2float(a)); }
};

template <class SIN, class LNK>
struct half_pair {
  static constexpr bool value = false;
};
template <class FMT>
struct half_pair<SpinorN16<FMT>, Link16<FMT>> {
  static constexpr bool value = QXD_HOP16_HMATH != 0;
  typedef FMT fmt;
};
// (not the staged link tile of the 16-bit multi-RHS hop: its per-(site, RHS) threads measured slower
// with the packed leg, 415 us against 390 us per launch on 24^3x48)

// One leg of a 16-bit hop in packed 16-bit arithmetic: the stored (unscaled) neighbour spinor is
// projected and multiplied by the stored link without conversion, i z = (-z.im, z.re) as a swap of
// the halves with a sign pair, every product a packed fused multiply-add; the transported half
// spinor is then widened to FP32 and accumulated with the per-site norm and the time sign.  Stored
// values lie in [-1, 1] (spinors divided by their site norm, unitary links), so no intermediate
// can leave the format's range.
template <class FMT, int MU, bool FWD, bool G5IN>
__device__ __forceinline__ void leg_half(const typename SpinorN16<FMT>::Raw& sr, const uint32_t lw[9], float sc,
                                         cplx<float> acc[12]) {
  typedef HM<FMT> H;
  typedef typename H::T T;
  const T NP = H::two(-1.f, 1.f), PN = H::two(1.f, -1.f);
  T s[12];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    s[2 * j] = H::word(sr.v[j].x);
    s[2 * j + 1] = H::word(sr.v[j].y);
  }
  // dn enters with the sign of gamma5 (G5IN) and of the projector
  auto pm = [](T a, T b, bool plus) { return plus ? __hadd2(a, b) : __hsub2(a, b); };
  auto pmi = [&](T a, T b, bool plus) { return __hfma2(__lowhigh2highlow(b), plus ? NP : PN, a); };  // a +- i b
  T h[6];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T up0 = s[c], up1 = s[3 + c], dn0 = s[6 + c], dn1 = s[9 + c];
    const bool f = FWD != G5IN;  // the sign of dn
    if (MU == 0) {
      h[c] = pm(up0, dn0, f);
      h[3 + c] = pm(up1, dn1, f);
    } else if (MU == 1) {
      h[c] = pmi(up0, dn1, f);
      h[3 + c] = pmi(up1, dn0, f);
    } else if (MU == 2) {
      h[c] = pm(up0, dn1, f);
      h[3 + c] = pm(up1, dn0, !f);
    } else {
      h[c] = pmi(up0, dn0, f);
      h[3 + c] = pmi(up1, dn1, !f);
    }
  }
  // t = W h (forward) or W^+ h (backward): u x = u.re x + (-u.im, u.im) swap(x),
  // conj(u) x = u.re x + (u.im, -u.im) swap(x)
  T t[6];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const T u = H::word(FWD ? lw[3 * a + b] : lw[3 * b + a]);
      const T ur = H::lo2(u), ui = __hmul2(H::hi2(u), FWD ? NP : PN);
#pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
        const T x = h[3 * sp + b];
        T& y = t[3 * sp + a];
        y = b == 0 ? __hmul2(ur, x) : __hfma2(ur, x, y);
        y = __hfma2(ui, __lowhigh2highlow(x), y);
      }
    }
  cplx<float> g[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) g[k] = H::f32(t[k]);
  accumulate_s<float, MU, FWD>(acc, g, sc);
}

template <int LEG, int PF, typename R, class SIN, class LNK, bool G5IN>
__device__ __forceinline__ void leg_step(const Geom& g, int par, uint32_t cb, const uint32_t nb[8], bool cr_f,
                                         bool cr_b, const SIN& in, const LNK& lk, typename SIN::Raw* sr,
                                         typename LNK::Raw* lr, cplx<R> acc[12]) {
  constexpr int MU = LEG >> 1;
  constexpr bool FWD = (LEG & 1) == 0;
  constexpr int slot = LEG % PF;
  if constexpr (half_pair<SIN, LNK>::value) {
    const typename SIN::Raw sraw = sr[slot];
    const typename LNK::Raw lraw = lr[slot];
    if constexpr (LEG + PF < 8) {
      constexpr int nl = LEG + PF;
      sr[slot] = in.fetch(nb[nl]);
      lr[slot] = lk.fetch((nl & 1) ? 1 - par : par, nl >> 1, (nl & 1) ? nb[nl] : cb);
    }
    float sc = sraw.n;
    if (MU == 0 && (FWD ? cr_f : cr_b) && g.anti) sc = -sc;
    uint32_t lw[9];
    lk.words(lraw, lw);
    leg_half<typename half_pair<SIN, LNK>::fmt, MU, FWD, G5IN>(sraw, lw, sc, acc);
    return;
  }
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
  link_mul<R, !FWD>(u, h, t);
  accumulate_s<R, MU, FWD>(acc, t, sc);
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
