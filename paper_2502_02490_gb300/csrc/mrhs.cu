// Multi-right-hand-side hop (FP32): one link and clover load serves R right-hand sides.
//
// A block covers 32 consecutive output sites (threadIdx.x) times up to 12 right-hand sides
// (threadIdx.y; rows beyond the launch's count only help load).  Phase 1: 256 threads compute the
// 8 neighbour indices of the 32 sites into shared memory.  Phase 2: the block loads the 32 sites' 8 links (forward links of the sites,
// backward links of their neighbours) and, when the epilogue needs it, the clover block pair
// into shared memory, coalesced across sites.  Phase 3: every thread applies the hop for its
// (site, rhs) with links and clover from shared memory and its neighbour spinors from global
// memory (L1/L2 serve the reuse).  Per site and RHS the algorithmic traffic is the spinors
// (in, out, diagonal in) plus (8 links + clover) / R.
#include <cstdlib>

#include "hop_site.cuh"

namespace qxd {

constexpr int MR_SITES = 32;
constexpr int MR_MAXR = 12;

struct MrShared {
  uint32_t nb[8][MR_SITES];
  unsigned char cross[2][MR_SITES];  // time-boundary crossing of the forward / backward t hop
  float2 link[8][9][MR_SITES];
  float4 clov[2][9][MR_SITES];
};

template <int LEG, bool G5IN>
__device__ __forceinline__ void mr_leg(const Geom& g, const MrShared& sh, int s, const float4* __restrict__ in,
                                       i64 sv, cplx<float> acc[12]) {
  constexpr int MU = LEG >> 1;
  constexpr bool FWD = (LEG & 1) == 0;
  const uint32_t n = sh.nb[LEG][s];
  cplx<float> v[12], h[6], u[9], t[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float4 q = __ldg(in + j * sv + n);
    v[2 * j] = mk(q.x, q.y);
    v[2 * j + 1] = mk(q.z, q.w);
  }
  if (G5IN) {
#pragma unroll
    for (int k = 6; k < 12; ++k) v[k] = neg(v[k]);
  }
  project<float, MU, FWD>(v, h);
  if (MU == 0 && g.anti && sh.cross[FWD ? 0 : 1][s]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = neg(h[k]);
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float2 w = sh.link[LEG][k][s];
    u[k] = mk(w.x, w.y);
  }
  link_mul<float, !FWD>(u, h, t);
  accumulate<float, MU, FWD>(acc, t);
}

__device__ __forceinline__ void mr_clover(const MrShared& sh, int s, const cplx<float> v[12], cplx<float> y[12]) {
#pragma unroll
  for (int blk = 0; blk < 2; ++blk) {
    float r[36];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float4 c = sh.clov[blk][k][s];
      r[4 * k] = c.x;
      r[4 * k + 1] = c.y;
      r[4 * k + 2] = c.z;
      r[4 * k + 3] = c.w;
    }
    herm6_apply<float>(r, v + 6 * blk, y + 6 * blk);
  }
}

// in/same/out: multi-RHS fields, RHS r of parity (1-par)/par/par at base + r * rs (float4s)
template <int EPI, bool G5>
__global__ void __launch_bounds__(MR_SITES* MR_MAXR, 2) k_hop_mrhs(Geom g, int par, int nr, const float4* __restrict__ in,
                                                               const float4* __restrict__ same, float4* __restrict__ out,
                                                               i64 rs, const float2* __restrict__ W,
                                                               const float4* __restrict__ C, float coef) {
  __shared__ MrShared sh;
  const int s = threadIdx.x, r = threadIdx.y;
  constexpr int NTHR = MR_SITES * MR_MAXR;  // the block always has MR_MAXR rows; rows >= nr only load
  const int tid = r * MR_SITES + s, nthr = NTHR;
  const uint32_t cb0 = blockIdx.x * MR_SITES;
  // phase 1: neighbour table (legs unrolled: register-only index math)
  for (int ss = tid; ss < MR_SITES; ss += nthr) {
    const uint32_t cb = cb0 + ss;
    const bool live = cb < (uint32_t)g.Vh;
    int x[4] = {0, 0, 0, 0};
    if (live) cb_coords32(g, cb, par, x);
#pragma unroll
    for (int leg = 0; leg < 8; ++leg) {
      bool cr = false;
      const uint32_t nbv = live ? nbr_cb32(g, x, leg >> 1, (leg & 1) ? -1 : +1, cr) : 0u;
      sh.nb[leg][ss] = nbv;
      if (leg < 2) sh.cross[leg][ss] = cr && live;
    }
  }
  __syncthreads();
  // phase 2: links (and clover), every load of a thread issued before its first shared store
  // (compile-time trip counts): one memory round trip per block
  constexpr int NL = (8 * 9 * MR_SITES + NTHR - 1) / NTHR;
  constexpr bool NEEDC = EPI != EPI_HOP && EPI != EPI_XPAY;
  constexpr int NC = NEEDC ? (2 * 9 * MR_SITES + NTHR - 1) / NTHR : 0;
  float2 wl[NL];
  float4 cvl[NC > 0 ? NC : 1];
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const int e = tid + i * NTHR;
    const int ss = e % MR_SITES, rest = e / MR_SITES, leg = rest / 9, k = rest % 9;
    const uint32_t cb = cb0 + ss;
    wl[i] = make_float2(0.f, 0.f);
    if (e < 8 * 9 * MR_SITES && cb < (uint32_t)g.Vh) {
      const int mu = leg >> 1;
      const bool fwd = (leg & 1) == 0;
      const int lp = fwd ? par : 1 - par;
      const uint32_t site = fwd ? cb : sh.nb[leg][ss];
      wl[i] = __ldg(W + ((i64)(lp * 4 + mu) * 9 + k) * g.sv + site);
    }
  }
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    const int e = tid + i * NTHR;
    const int ss = e % MR_SITES, rest = e / MR_SITES, blk = rest / 9, k = rest % 9;
    const uint32_t cb = cb0 + ss;
    cvl[i] = (e < 2 * 9 * MR_SITES && cb < (uint32_t)g.Vh) ? __ldg(C + ((i64)(par * 2 + blk) * 9 + k) * g.sv + cb)
                                                          : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const int e = tid + i * NTHR;
    if (e < 8 * 9 * MR_SITES) sh.link[(e / MR_SITES) / 9][(e / MR_SITES) % 9][e % MR_SITES] = wl[i];
  }
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    const int e = tid + i * NTHR;
    if (e < 2 * 9 * MR_SITES) sh.clov[(e / MR_SITES) / 9][(e / MR_SITES) % 9][e % MR_SITES] = cvl[i];
  }
  __syncthreads();
  const uint32_t cb = cb0 + s;
  if (cb >= (uint32_t)g.Vh || r >= nr) return;
  const float4* inr = in + r * rs;
  cplx<float> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = mk(0.f, 0.f);
  constexpr bool G5IN = G5 && EPI == EPI_INV;
  mr_leg<0, G5IN>(g, sh, s, inr, g.sv, acc);
  mr_leg<1, G5IN>(g, sh, s, inr, g.sv, acc);
  mr_leg<2, G5IN>(g, sh, s, inr, g.sv, acc);
  mr_leg<3, G5IN>(g, sh, s, inr, g.sv, acc);
  mr_leg<4, G5IN>(g, sh, s, inr, g.sv, acc);
  mr_leg<5, G5IN>(g, sh, s, inr, g.sv, acc);
  mr_leg<6, G5IN>(g, sh, s, inr, g.sv, acc);
  mr_leg<7, G5IN>(g, sh, s, inr, g.sv, acc);
  auto load = [&](const float4* f, cplx<float> v[12]) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float4 q = __ldg(f + r * rs + j * g.sv + cb);
      v[2 * j] = mk(q.x, q.y);
      v[2 * j + 1] = mk(q.z, q.w);
    }
  };
  cplx<float> o[12];
  if (EPI == EPI_HOP) {
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = coef * acc[k];
  } else if (EPI == EPI_DFULL || EPI == EPI_DHAT2) {
    cplx<float> v[12], y[12];
    load(same, v);
    mr_clover(sh, s, v, y);
    const float c = EPI == EPI_DFULL ? -0.5f : coef;
    if (EPI == EPI_DHAT2 && G5) {
#pragma unroll
      for (int k = 6; k < 12; ++k) acc[k] = neg(acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = y[k] + c * acc[k];
  } else if (EPI == EPI_INV) {
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = coef * acc[k];
    mr_clover(sh, s, acc, o);
  } else if (EPI == EPI_INVXPAY) {
    cplx<float> v[12];
    load(same, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = v[k] + coef * acc[k];
    mr_clover(sh, s, v, o);
  } else {  // EPI_XPAY
    cplx<float> v[12];
    load(same, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = v[k] + coef * acc[k];
  }
  float4* outr = out + r * rs;
#pragma unroll
  for (int j = 0; j < 6; ++j) outr[j * g.sv + cb] = make_float4(o[2 * j].re, o[2 * j].im, o[2 * j + 1].re, o[2 * j + 1].im);
}

qxd_status hop32_mrhs(qxd_lattice* lat, int par, int epi, int g5, const float4* in, const float4* same, float4* out,
                      float coef, int nrhs, i64 rs) {
  const Geom& g = lat->g;
  for (int r0 = 0; r0 < nrhs; r0 += MR_MAXR) {
    const int nr = nrhs - r0 < MR_MAXR ? nrhs - r0 : MR_MAXR;
    dim3 grid((unsigned)((g.Vh + MR_SITES - 1) / MR_SITES)), block(MR_SITES, MR_MAXR);  // rows >= nr only load
    const float4* i0 = in + r0 * rs;
    const float4* s0 = same ? same + r0 * rs : nullptr;
    float4* o0 = out + r0 * rs;
    const float4* C = (epi == EPI_INV || epi == EPI_INVXPAY) ? lat->Ci32 : lat->C32;
    // bytes: per site and RHS the spinors; links and clover once per site for the whole block
    double sp = 96.0 * (2 + ((epi == EPI_DFULL || epi == EPI_DHAT2 || epi == EPI_INVXPAY || epi == EPI_XPAY) ? 1 : 0));
    double once = 8 * 72.0 + ((epi != EPI_HOP && epi != EPI_XPAY) ? 288.0 : 0.0);
    prof_begin(lat, KSTAT_F32_MRHS, (sp * nr + once) * (double)g.Vh);
#define QXD_MR_CASE(E, G) \
  if (epi == E && (g5 != 0) == G) k_hop_mrhs<E, G><<<grid, block, 0, lat->stream>>>(g, par, nr, i0, s0, o0, rs, lat->W32, C, coef); else
    QXD_MR_CASE(EPI_HOP, false)
    QXD_MR_CASE(EPI_DFULL, false)
    QXD_MR_CASE(EPI_INV, false)
    QXD_MR_CASE(EPI_INV, true)
    QXD_MR_CASE(EPI_DHAT2, false)
    QXD_MR_CASE(EPI_DHAT2, true)
    QXD_MR_CASE(EPI_XPAY, false)
    QXD_MR_CASE(EPI_INVXPAY, false) {
      prof_end(lat);
      return fail(lat, QXD_EINVAL, "unsupported multi-RHS epilogue");
    }
#undef QXD_MR_CASE
    prof_end(lat);
    QXD_CHECK_LAUNCH(lat, "k_hop_mrhs");
  }
  return QXD_OK;
}

// ------------------------------------------------------------------------------------------
// 16-bit multi-RHS hop.  Spinors of each right-hand side in 16 bits with a per-site FP32 norm
// (as the single-RHS 16-bit hop); links and the clover block pair of a tile of MR16_SITES
// sites are staged once in shared memory (16-bit, as stored) and serve the NRB right-hand
// sides of the block.  A block is MR16_SITES sites (threadIdx.x, one warp per right-hand side)
// times NRB right-hand sides (threadIdx.y); blockIdx.y selects a group of NRB right-hand sides.
// Each thread runs the software-pipelined hop of the single-RHS kernel (neighbour spinors
// fetched PF legs ahead) with its link and clover reads served by shared memory.  Per site and
// RHS the algorithmic bytes are the spinors (52 B each: in, out, diagonal in) plus
// (8 x 36 B links + 152 B clover) / NRB.
// ------------------------------------------------------------------------------------------
constexpr int MR16_SITES = 32;

template <int S>
struct Mr16Shared {
  uint32_t nbb[4][S];      // backward neighbours (cb in the other parity) of the tile's sites
  uint32_t link[8][9][S];  // leg 2 mu: W_mu(x); leg 2 mu + 1: W_mu(x - mu) (16-bit pairs)
  uint2 clov[2][9][S];     // clover block pair (16-bit) and its per-block norms
  float cn[2][S];
};

// Link accessor over the staged tile: a "raw" link is only the leg; decode reads shared memory.
template <class FMT, int S>
struct LinkTile16 {
  typedef float real;
  struct Raw {
    int leg;
  };
  const Mr16Shared<S>* sh;
  int s, par;
  __device__ __forceinline__ Raw fetch(int lp, int mu, uint32_t) const { return Raw{2 * mu + (lp != par ? 1 : 0)}; }
  __device__ __forceinline__ void decode(const Raw& r, cplx<float> u[9]) const {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const uint32_t w = sh->link[r.leg][k][s];
      u[k] = mk(FMT::lo(w), FMT::hi(w));
    }
  }
};

// Clover accessor over the staged tile (the epilogue reads it when it needs it).
template <class FMT, int S>
struct CloverTile16 {
  typedef float real;
  struct Raw {};
  const Mr16Shared<S>* sh;
  int s;
  __device__ __forceinline__ Raw fetch(int, uint32_t) const { return Raw{}; }
  __device__ __forceinline__ void decode(const Raw&, int blk, float o[36]) const {
    const float n = sh->cn[blk][s];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const uint2 v = sh->clov[blk][k][s];
      o[4 * k] = n * FMT::lo(v.x);
      o[4 * k + 1] = n * FMT::hi(v.x);
      o[4 * k + 2] = n * FMT::lo(v.y);
      o[4 * k + 3] = n * FMT::hi(v.y);
    }
  }
};
template <class F, int S>
struct is16<CloverTile16<F, S>> {
  static constexpr bool value = true;  // epilogue data prefetched like the 16-bit single-RHS hop
};

template <class FMT, int NRB, int MINB, bool OUT16, int EPI, bool G5>
__global__ void __launch_bounds__(MR16_SITES* NRB, MINB)
    k_hop_mrhs16(Geom g, int par, int nr, const uint2* __restrict__ in, const float* __restrict__ in_n,
                 const uint2* __restrict__ same, const float* __restrict__ same_n, uint2* __restrict__ out,
                 float* __restrict__ out_n, float4* __restrict__ out32, const uint32_t* __restrict__ W,
                 const uint2* __restrict__ C, const float* __restrict__ Cn, float coef) {
  constexpr int S = MR16_SITES;
  __shared__ Mr16Shared<S> sh;
  const int s = threadIdx.x, rb = threadIdx.y;
  const int tid = rb * S + s, nthr = S * NRB;
  const uint32_t cb0 = blockIdx.x * S;
  const i64 sv = g.sv;
  (void)nthr;
  // phase 1: backward neighbours of the tile (directions unrolled: register-only index math)
  for (int ss = tid; ss < S; ss += nthr) {
    const uint32_t cb = cb0 + ss;
    int x[4] = {0, 0, 0, 0};
    const bool live = cb < (uint32_t)g.Vh;
    if (live) cb_coords32(g, cb, par, x);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      bool cr;
      sh.nbb[mu][ss] = live ? nbr_cb32(g, x, mu, -1, cr) : 0u;
    }
  }
  __syncthreads();
  // phase 2: the tile's links and clover (coalesced across sites).  The trip counts are compile-
  // time constants so that every load of a thread is issued before the first store to shared
  // memory: one memory round trip per block instead of one per loop iteration.
  constexpr int NTHR = S * NRB;
  constexpr int NL = (8 * 9 * S + NTHR - 1) / NTHR;
  constexpr bool NEEDC = EPI != EPI_HOP && EPI != EPI_XPAY;
  constexpr int NC = NEEDC ? (2 * 9 * S + NTHR - 1) / NTHR : 0;
  constexpr int NN = NEEDC ? (2 * S + NTHR - 1) / NTHR : 0;
  uint32_t wl[NL];
  uint2 cvl[NC > 0 ? NC : 1];
  float cnl[NN > 0 ? NN : 1];
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const int e = tid + i * NTHR;
    const int ss = e % S, rest = e / S, leg = rest / 9, k = rest % 9;
    const uint32_t cb = cb0 + ss;
    wl[i] = 0u;
    if (e < 8 * 9 * S && cb < (uint32_t)g.Vh) {
      const int mu = leg >> 1;
      const bool fwd = (leg & 1) == 0;
      const int lp = fwd ? par : 1 - par;
      wl[i] = __ldg(W + ((i64)(lp * 4 + mu) * 9 + k) * sv + (fwd ? cb : sh.nbb[mu][ss]));
    }
  }
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    const int e = tid + i * NTHR;
    const int ss = e % S, rest = e / S, blk = rest / 9, k = rest % 9;
    const uint32_t cb = cb0 + ss;
    cvl[i] = (e < 2 * 9 * S && cb < (uint32_t)g.Vh) ? __ldg(C + ((i64)(par * 2 + blk) * 9 + k) * sv + cb)
                                                 : make_uint2(0u, 0u);
  }
#pragma unroll
  for (int i = 0; i < NN; ++i) {
    const int e = tid + i * NTHR;
    const int ss = e % S, blk = e / S;
    const uint32_t cb = cb0 + ss;
    cnl[i] = (e < 2 * S && cb < (uint32_t)g.Vh) ? __ldg(Cn + (i64)(par * 2 + blk) * sv + cb) : 0.f;
  }
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const int e = tid + i * NTHR;
    if (e < 8 * 9 * S) sh.link[(e / S) / 9][(e / S) % 9][e % S] = wl[i];
  }
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    const int e = tid + i * NTHR;
    if (e < 2 * 9 * S) sh.clov[(e / S) / 9][(e / S) % 9][e % S] = cvl[i];
  }
#pragma unroll
  for (int i = 0; i < NN; ++i) {
    const int e = tid + i * NTHR;
    if (e < 2 * S) sh.cn[e / S][e % S] = cnl[i];
  }
  __syncthreads();
  const uint32_t cb = cb0 + s;
  const int r = blockIdx.y * NRB + rb;
  if (cb >= (uint32_t)g.Vh || r >= nr) return;
  const i64 o16 = (i64)r * 6 * sv, on = (i64)r * sv;
  SpinorN16<FMT> si{const_cast<uint2*>(in) + o16, const_cast<float*>(in_n) + on, sv};
  SpinorN16<FMT> ssame{const_cast<uint2*>(same) + (same ? o16 : 0), const_cast<float*>(same_n) + (same_n ? on : 0), sv};
  LinkTile16<FMT, S> lk{&sh, s, par};
  CloverTile16<FMT, S> cl{&sh, s};
  if constexpr (OUT16) {
    SpinorN16<FMT> so{out + o16, out_n + on, sv};
    hop_site<float, SpinorN16<FMT>, SpinorN16<FMT>, SpinorN16<FMT>, LinkTile16<FMT, S>, CloverTile16<FMT, S>, EPI, G5,
             QXD_HOP_PF16>(g, par, cb, si, ssame, so, lk, cl, coef);
  } else {
    SpinorF32 so{out32 + o16, sv};
    hop_site<float, SpinorN16<FMT>, SpinorN16<FMT>, SpinorF32, LinkTile16<FMT, S>, CloverTile16<FMT, S>, EPI, G5,
             QXD_HOP_PF16>(g, par, cb, si, ssame, so, lk, cl, coef);
  }
}

// Right-hand sides per block of the 16-bit multi-RHS hop: 12, 6 or 4 (the environment variable
// QXD_MRHS16_NRB overrides the default, for shape sweeps).
static int mrhs16_nrb() {
  static int nrb = [] {
    const char* e = std::getenv("QXD_MRHS16_NRB");
    int v = e ? std::atoi(e) : 6;
    return (v == 12 || v == 6 || v == 4) ? v : 6;
  }();
  return nrb;
}

template <class FMT, int NRB, int MINB, bool OUT16>
static qxd_status launch_mrhs16(qxd_lattice* lat, int par, int epi, int g5, const uint2* in, const float* in_n,
                                const uint2* same, const float* same_n, uint2* out, float* out_n, float4* out32,
                                const uint32_t* W, const uint2* C, const float* Cn, float coef, int nrhs) {
  const Geom& g = lat->g;
  dim3 grid((unsigned)((g.Vh + MR16_SITES - 1) / MR16_SITES), (unsigned)((nrhs + NRB - 1) / NRB)),
      block(MR16_SITES, NRB);
#define QXD_MR16_CASE(E, G)                                                                                        \
  if (epi == E && (g5 != 0) == G)                                                                                  \
    k_hop_mrhs16<FMT, NRB, MINB, OUT16, E, G><<<grid, block, 0, lat->stream>>>(g, par, nrhs, in, in_n, same, same_n, \
                                                                              out, out_n, out32, W, C, Cn, coef);   \
  else
  QXD_MR16_CASE(EPI_INV, false)
  QXD_MR16_CASE(EPI_INV, true)
  QXD_MR16_CASE(EPI_DHAT2, false)
  QXD_MR16_CASE(EPI_DHAT2, true)
  QXD_MR16_CASE(EPI_DFULL, false) { return fail(lat, QXD_EINVAL, "unsupported 16-bit multi-RHS epilogue"); }
#undef QXD_MR16_CASE
  QXD_CHECK_LAUNCH(lat, "k_hop_mrhs16");
  return QXD_OK;
}

template <class FMT, bool OUT16>
static qxd_status mrhs16_shape(qxd_lattice* lat, int par, int epi, int g5, const uint2* in, const float* in_n,
                               const uint2* same, const float* same_n, uint2* out, float* out_n, float4* out32,
                               const uint32_t* W, const uint2* C, const float* Cn, float coef, int nrhs) {
  switch (mrhs16_nrb()) {
    case 12:
      return launch_mrhs16<FMT, 12, 2, OUT16>(lat, par, epi, g5, in, in_n, same, same_n, out, out_n, out32, W, C, Cn,
                                              coef, nrhs);
    case 4:
      return launch_mrhs16<FMT, 4, 5, OUT16>(lat, par, epi, g5, in, in_n, same, same_n, out, out_n, out32, W, C, Cn,
                                             coef, nrhs);
    default:
      return launch_mrhs16<FMT, 6, 3, OUT16>(lat, par, epi, g5, in, in_n, same, same_n, out, out_n, out32, W, C, Cn,
                                             coef, nrhs);
  }
}

qxd_status hop16_mrhs(qxd_lattice* lat, int bf16, int par, int epi, int g5, const uint2* in, const float* in_nrm,
                      const uint2* same, const float* same_nrm, uint2* out, float* out_nrm, float4* out32, float coef,
                      int nrhs) {
  if (nrhs < 1) return fail(lat, QXD_EINVAL, "nrhs must be positive");
  if (!out32 && !(out && out_nrm)) return fail(lat, QXD_EINVAL, "16-bit multi-RHS hop: no output");
  const bool inv = epi == EPI_INV || epi == EPI_INVXPAY;
  const bool needs_same = epi == EPI_DFULL || epi == EPI_DHAT2;
  if (needs_same && !(same && same_nrm)) return fail(lat, QXD_EINVAL, "16-bit multi-RHS hop: epilogue needs same");
  const Geom& g = lat->g;
  const int nrb = mrhs16_nrb();
  // bytes: per site and RHS the spinors; links and clover once per site and block of nrb RHS
  const double sp = 52.0 + (out32 ? 96.0 : 52.0) + (needs_same ? 52.0 : 0.0);
  const double groups = (double)((nrhs + nrb - 1) / nrb);
  prof_begin(lat, KSTAT_N16_MRHS, (sp * nrhs + groups * (8 * 36.0 + 152.0)) * (double)g.Vh);
  qxd_status st;
  if (bf16) {
    const uint32_t* W = lat->WB16;
    const uint2* C = inv ? lat->CiB16 : lat->CB16;
    const float* Cn = inv ? lat->CiB16n : lat->CB16n;
    st = out32 ? mrhs16_shape<B16, false>(lat, par, epi, g5, in, in_nrm, same, same_nrm, out, out_nrm, out32, W, C, Cn,
                                          coef, nrhs)
               : mrhs16_shape<B16, true>(lat, par, epi, g5, in, in_nrm, same, same_nrm, out, out_nrm, out32, W, C, Cn,
                                         coef, nrhs);
  } else {
    const uint32_t* W = lat->W16;
    const uint2* C = inv ? lat->Ci16 : lat->C16;
    const float* Cn = inv ? lat->Ci16n : lat->C16n;
    st = out32 ? mrhs16_shape<H16, false>(lat, par, epi, g5, in, in_nrm, same, same_nrm, out, out_nrm, out32, W, C, Cn,
                                          coef, nrhs)
               : mrhs16_shape<H16, true>(lat, par, epi, g5, in, in_nrm, same, same_nrm, out, out_nrm, out32, W, C, Cn,
                                         coef, nrhs);
  }
  prof_end(lat);
  return st;
}

}  // namespace qxd
