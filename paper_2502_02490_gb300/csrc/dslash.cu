// The hopping term (dslash) of the Wilson-clover operator with fused clover epilogues.
//
// (H psi)(x) = sum_mu [(1 - gamma_mu) W_mu(x) psi(x+mu) + (1 + gamma_mu) W_mu(x-mu)^dag psi(x-mu)]
// (the hop part of the method's operator; D = A - H/2, Sec. 1-2 and Sec. 4.3 for U(3) links W).
//
// Spin projection in the chiral basis (gamma_0 = [[0,-1],[-1,0]], gamma_k = [[0,-i s_k],[i s_k,0]]):
//   (1 -+ gamma_0) psi = [h; +-h]        with h = up +- dn
//   (1 -+ gamma_k) psi = [h; -+ i s_k h] with h = up +- i s_k dn
// (up = spins 0,1; dn = spins 2,3), so each direction moves a 2-spin x 3-colour half spinor
// through one 3x3 link multiply.  One thread per output site; the neighbour spinors come from
// the opposite parity.  Time-boundary sign and C* neighbours follow nbr_cb().
#include "hop_common.cuh"

namespace qxd {

// One of the eight hops ("legs": 2*mu + 0 forward, 2*mu + 1 backward) of the software-pipelined
// kernel: decode the raw neighbour spinor and link fetched PF legs earlier, refill the slot with
// the raw data of leg LEG + PF, then project, scale (per-site norm and time-boundary sign, applied
// once to the 6-component half spinor), transport and accumulate.
constexpr int HOP_BLOCK = 128;
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

// (Norms of the output are taken by a separate BLAS pass: a block reduction inside this
// latency-bound kernel measured slower on GB300 than the extra bandwidth-bound pass.)
template <typename R, class SIN, class SSAME, class SOUT, class LNK, class CLV, int EPI, bool G5, int PF>
__global__ void __launch_bounds__(HOP_BLOCK, is16<CLV>::value ? QXD_HOP16_MINB : 1) k_hop(Geom g, int par, SIN in, SSAME same, SOUT out, LNK lk, CLV cl,
                                                   R coef) {
  const uint32_t cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= (uint32_t)g.Vh) return;
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
  constexpr bool G5IN = G5 && (EPI == EPI_INV);
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
    if (EPI == EPI_DHAT2 && G5) {
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
}

// Algorithmic bytes of one launch (per output site: neighbour spinors counted once, 8 links,
// the clover block pair, the diagonal input where used, the output).
static double hop_bytes(qxd_lattice* lat, int epi, double sp_in, double sp_out, double link, double clov) {
  double b = sp_in + sp_out + 8 * link;
  if (epi != EPI_HOP && epi != EPI_XPAY) b += clov;
  if (epi == EPI_DFULL || epi == EPI_DHAT2 || epi == EPI_INVXPAY || epi == EPI_XPAY) b += sp_in;
  return b * (double)lat->Vh;
}

template <typename R, int PF, class SIN, class SSAME, class SOUT, class LNK, class CLV>
static qxd_status launch_hop(qxd_lattice* lat, int par, int epi, int g5, SIN in, SSAME same, SOUT out, LNK lk,
                             CLV cl, R coef) {
  const Geom& g = lat->g;
  dim3 grid(grid_for(g.Vh, HOP_BLOCK)), block(HOP_BLOCK);
  cudaStream_t st = lat->stream;
#define QXD_HOP_CASE(E, G)                                                                                  \
  if (epi == E && (g5 != 0) == G) {                                                                         \
    k_hop<R, SIN, SSAME, SOUT, LNK, CLV, E, G, PF><<<grid, block, 0, st>>>(g, par, in, same, out, lk, cl, coef); \
  } else
  QXD_HOP_CASE(EPI_HOP, false)
  QXD_HOP_CASE(EPI_DFULL, false)
  QXD_HOP_CASE(EPI_INV, false)
  QXD_HOP_CASE(EPI_INV, true)
  QXD_HOP_CASE(EPI_DHAT2, false)
  QXD_HOP_CASE(EPI_DHAT2, true)
  QXD_HOP_CASE(EPI_XPAY, false)
  QXD_HOP_CASE(EPI_INVXPAY, false) { return fail(lat, QXD_EINVAL, "unsupported hop epilogue"); }
#undef QXD_HOP_CASE
  QXD_CHECK_LAUNCH(lat, "k_hop");
  return QXD_OK;
}

qxd_status hop64(qxd_lattice* lat, int par, int epi, int g5, const double2* in, const double2* same, double2* out,
                 double coef) {
  const i64 sv = lat->sv;
  SpinorF64 si{const_cast<double2*>(in), sv}, ss{const_cast<double2*>(same), sv}, so{out, sv};
  LinkF64 lk{lat->W64, sv};
  bool inv = epi == EPI_INV || epi == EPI_INVXPAY;
  CloverF64 cl{inv ? lat->Ci64 : lat->C64, sv};
  prof_begin(lat, KSTAT_F64, hop_bytes(lat, epi, 192, 192, 144, 576));
  qxd_status st = launch_hop<double, 2>(lat, par, epi, g5, si, ss, so, lk, cl, coef);
  prof_end(lat);
  return st;
}

qxd_status hop32(qxd_lattice* lat, int par, int epi, int g5, const float4* in, const float4* same, float4* out,
                 float coef) {
  const i64 sv = lat->sv;
  SpinorF32 si{const_cast<float4*>(in), sv}, ss{const_cast<float4*>(same), sv}, so{out, sv};
  LinkF32 lk{lat->W32, sv};
  bool inv = epi == EPI_INV || epi == EPI_INVXPAY;
  CloverF32 cl{inv ? lat->Ci32 : lat->C32, sv};
  prof_begin(lat, KSTAT_F32, hop_bytes(lat, epi, 96, 96, 72, 288));
  qxd_status st = launch_hop<float, 2>(lat, par, epi, g5, si, ss, so, lk, cl, coef);
  prof_end(lat);
  return st;
}

template <class FMT>
static qxd_status hop16_t(qxd_lattice* lat, int kind, int par, int epi, int g5, const uint2* in, const float* in_nrm,
                          const uint2* same, const float* same_nrm, uint2* out, float* out_nrm, float4* out32,
                          float coef, const uint32_t* W, const uint2* C, const float* Cn) {
  const i64 sv = lat->sv;
  SpinorN16<FMT> si{const_cast<uint2*>(in), const_cast<float*>(in_nrm), sv};
  SpinorN16<FMT> ss{const_cast<uint2*>(same), const_cast<float*>(same_nrm), sv};
  Link16<FMT> lk{W, sv};
  Clover16<FMT> cl{C, Cn, sv};
  double bytes;
  qxd_status st;
  if (out32) {
    SpinorF32 so{out32, sv};
    bytes = hop_bytes(lat, epi, 52, 96, 36, 152);
    prof_begin(lat, kind, bytes);
    st = launch_hop<float, QXD_HOP_PF16>(lat, par, epi, g5, si, ss, so, lk, cl, coef);
  } else {
    SpinorN16<FMT> so{out, out_nrm, sv};
    bytes = hop_bytes(lat, epi, 52, 52, 36, 152);
    prof_begin(lat, kind, bytes);
    st = launch_hop<float, QXD_HOP_PF16>(lat, par, epi, g5, si, ss, so, lk, cl, coef);
  }
  prof_end(lat);
  return st;
}

qxd_status hop16(qxd_lattice* lat, int bf16, int par, int epi, int g5, const uint2* in, const float* in_nrm,
                 const uint2* same, const float* same_nrm, uint2* out, float* out_nrm, float4* out32, float coef) {
  bool inv = epi == EPI_INV || epi == EPI_INVXPAY;
  if (bf16)
    return hop16_t<B16>(lat, KSTAT_BF16N, par, epi, g5, in, in_nrm, same, same_nrm, out, out_nrm, out32, coef,
                        lat->WB16, inv ? lat->CiB16 : lat->CB16, inv ? lat->CiB16n : lat->CB16n);
  return hop16_t<H16>(lat, KSTAT_F16N, par, epi, g5, in, in_nrm, same, same_nrm, out, out_nrm, out32, coef,
                      lat->W16, inv ? lat->Ci16 : lat->C16, inv ? lat->Ci16n : lat->C16n);
}

}  // namespace qxd
