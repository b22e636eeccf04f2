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
#include "hop_site.cuh"

namespace qxd {

constexpr int HOP_BLOCK = 128;

// (Norms of the output are taken by a separate BLAS pass: a block reduction inside this
// latency-bound kernel measured slower on GB300 than the extra bandwidth-bound pass.)
template <typename R, class SIN, class SSAME, class SOUT, class LNK, class CLV, int EPI, bool G5, int PF>
__global__ void __launch_bounds__(HOP_BLOCK, is16<CLV>::value ? QXD_HOP16_MINB : 1) k_hop(Geom g, int par, SIN in, SSAME same, SOUT out, LNK lk, CLV cl,
                                                   R coef) {
  const uint32_t cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= (uint32_t)g.Vh) return;
  hop_site<R, SIN, SSAME, SOUT, LNK, CLV, EPI, G5, PF>(g, par, cb, in, same, out, lk, cl, coef);
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
  QXD_HOP_CASE(EPI_DFULL, true)
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
