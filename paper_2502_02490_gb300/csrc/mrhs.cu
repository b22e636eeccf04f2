// Multi-right-hand-side hop (FP32): one link and clover load serves R right-hand sides.
//
// A block covers 32 consecutive output sites (threadIdx.x) times R right-hand sides
// (threadIdx.y).  Phase 1: 256 threads compute the 8 neighbour indices of the 32 sites into
// shared memory.  Phase 2: the block loads the 32 sites' 8 links (forward links of the sites,
// backward links of their neighbours) and, when the epilogue needs it, the clover block pair
// into shared memory, coalesced across sites.  Phase 3: every thread applies the hop for its
// (site, rhs) with links and clover from shared memory and its neighbour spinors from global
// memory (L1/L2 serve the reuse).  Per site and RHS the algorithmic traffic is the spinors
// (in, out, diagonal in) plus (8 links + clover) / R.
#include "hop_common.cuh"

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
  const int tid = r * MR_SITES + s, nthr = MR_SITES * nr;
  const uint32_t cb0 = blockIdx.x * MR_SITES;
  // phase 1: neighbour table
  for (int e = tid; e < 8 * MR_SITES; e += nthr) {
    const int ss = e % MR_SITES, leg = e / MR_SITES;
    const uint32_t cb = cb0 + ss;
    uint32_t nbv = 0;
    bool cr = false;
    if (cb < (uint32_t)g.Vh) {
      int x[4];
      cb_coords32(g, cb, par, x);
      nbv = nbr_cb32(g, x, leg >> 1, (leg & 1) ? -1 : +1, cr);
    }
    sh.nb[leg][ss] = nbv;
    if (leg == 0) sh.cross[0][ss] = cr;
    if (leg == 1) sh.cross[1][ss] = cr;
  }
  __syncthreads();
  // phase 2: links (and clover)
  for (int e = tid; e < 8 * 9 * MR_SITES; e += nthr) {
    const int ss = e % MR_SITES, rest = e / MR_SITES, leg = rest / 9, k = rest % 9;
    const uint32_t cb = cb0 + ss;
    float2 w = make_float2(0.f, 0.f);
    if (cb < (uint32_t)g.Vh) {
      const int mu = leg >> 1;
      const bool fwd = (leg & 1) == 0;
      const int lp = fwd ? par : 1 - par;
      const uint32_t site = fwd ? cb : sh.nb[leg][ss];
      w = __ldg(W + ((i64)(lp * 4 + mu) * 9 + k) * g.sv + site);
    }
    sh.link[leg][k][ss] = w;
  }
  constexpr bool NEEDC = EPI != EPI_HOP && EPI != EPI_XPAY;
  if (NEEDC) {
    for (int e = tid; e < 2 * 9 * MR_SITES; e += nthr) {
      const int ss = e % MR_SITES, rest = e / MR_SITES, blk = rest / 9, k = rest % 9;
      const uint32_t cb = cb0 + ss;
      sh.clov[blk][k][ss] =
          cb < (uint32_t)g.Vh ? __ldg(C + ((i64)(par * 2 + blk) * 9 + k) * g.sv + cb) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
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
    dim3 grid((unsigned)((g.Vh + MR_SITES - 1) / MR_SITES)), block(MR_SITES, nr);
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

}  // namespace qxd
