// Multi-right-hand-side hops: one link and clover load serves up to 12 right-hand sides.
//
// FP32: a persistent kernel over tile records (32 consecutive checkerboard sites with their 8
// neighbour indices, 8 links and clover block pair, stored contiguously); one bulk copy per tile
// stages the record in shared memory while the block computes the previous tile.  Every thread
// applies the hop for its (site, rhs) with links and clover from shared memory and its neighbour
// spinors from global memory (L1/L2 serve the reuse).  Per site and RHS the algorithmic traffic
// is the spinors (in, out, diagonal in) plus (8 links + clover) / R.
//
// 16 bits: spinors, links and clover with per-site FP32 norms (below).
#include <cstdlib>

#include "hop_site.cuh"
#include "tc_common.cuh"

namespace qxd {

constexpr int MR_MAXR = 12;

// The right-hand sides one launch works on: local row r of a block is right-hand side idx[r]
// (its fields at base + idx[r] * rs), so frozen right-hand sides cost no hop work.
struct MrList {
  int idx[MR_MAXR];
};

// ------------------------------------------------------------------------------------------
// Tile records of the FP32 multi-RHS hop.  For each parity and each tile of MT_S consecutive
// checkerboard sites one contiguous record holds everything the hop reads once per site:
//     [clover A: 2 x 9 x MT_S float4][neighbours: 8 x MT_S uint32][links: 8 x 9 x MT_S float2]
//     [A^-1: 2 x 9 x MT_S float4]
// Leg 2 mu holds W_mu(x) (applied as W), leg 2 mu + 1 holds W_mu(x - mu) (applied as W^+), so the
// backward links sit beside the site instead of at its neighbour.  A neighbour entry is the
// checkerboard index of x +- mu; bit 31 marks a time hop across the antiperiodic boundary.  A
// kernel stages the part it needs, [clover][neighbours][links] or [neighbours][links][A^-1], with
// one bulk copy.  Sites beyond Vh in the last tile are zero.  The records are rebuilt whenever
// the gauge field or the clover term changes (the lattice's epoch).
// ------------------------------------------------------------------------------------------
constexpr int MT_S = 32;
constexpr uint32_t MT_CLOV = 2 * 9 * MT_S * 16;
constexpr uint32_t MT_NB = 8 * MT_S * 4;
constexpr uint32_t MT_W = 8 * 9 * MT_S * 8;
constexpr uint32_t MT_OFF_NB = MT_CLOV, MT_OFF_W = MT_CLOV + MT_NB, MT_OFF_CI = MT_CLOV + MT_NB + MT_W;
constexpr uint32_t MT_REC = 2 * MT_CLOV + MT_NB + MT_W;
constexpr long long MT_WAIT = 1ll << 24;  // polls of a tile's mbarrier before the kernel gives up
enum { MW_TILES = 60, MW_TILE_ERR = 61 };

__global__ void k_mr_tiles(Geom g, int par, const float2* __restrict__ W, const float4* __restrict__ C,
                           const float4* __restrict__ Ci, unsigned char* __restrict__ rec0, i64 ntiles) {
  const i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x;
  if (e >= ntiles * MT_S) return;
  const i64 tile = e / MT_S, cb = e;
  const int s = (int)(e % MT_S);
  unsigned char* rec = rec0 + tile * MT_REC;
  float4* cl = (float4*)rec;
  uint32_t* nb = (uint32_t*)(rec + MT_OFF_NB);
  float2* wl = (float2*)(rec + MT_OFF_W);
  float4* ci = (float4*)(rec + MT_OFF_CI);
  const bool live = cb < g.Vh;
  int x[4] = {0, 0, 0, 0};
  if (live) cb_coords32(g, (uint32_t)cb, par, x);
#pragma unroll
  for (int leg = 0; leg < 8; ++leg) {
    const int mu = leg >> 1;
    const bool fwd = (leg & 1) == 0;
    bool cr = false;
    const uint32_t n = live ? nbr_cb32(g, x, mu, fwd ? +1 : -1, cr) : 0u;
    nb[leg * MT_S + s] = n | ((live && mu == 0 && g.anti && cr) ? 0x80000000u : 0u);
    const int lp = fwd ? par : 1 - par;
    const i64 site = fwd ? cb : (i64)n;
    for (int k = 0; k < 9; ++k)
      wl[(leg * 9 + k) * MT_S + s] = live ? W[((i64)(lp * 4 + mu) * 9 + k) * g.sv + site] : make_float2(0.f, 0.f);
  }
  for (int bk = 0; bk < 18; ++bk) {  // bk = blk * 9 + k
    const i64 src = ((i64)par * 18 + bk) * g.sv + cb;
    cl[bk * MT_S + s] = (live && C) ? C[src] : make_float4(0.f, 0.f, 0.f, 0.f);
    ci[bk * MT_S + s] = (live && Ci) ? Ci[src] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

template <int LEG, bool G5IN>
__device__ __forceinline__ void mt_leg(const uint32_t* __restrict__ nbt, const float2* __restrict__ wt, int s,
                                       const float4* __restrict__ in, i64 sv, cplx<float> acc[12]) {
  constexpr int MU = LEG >> 1;
  constexpr bool FWD = (LEG & 1) == 0;
  const uint32_t e = nbt[LEG * MT_S + s];
  const uint32_t n = e & 0x7fffffffu;
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
  if (MU == 0 && (e >> 31)) {
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = neg(h[k]);
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float2 w = wt[(LEG * 9 + k) * MT_S + s];
    u[k] = mk(w.x, w.y);
  }
  link_mul<float, !FWD>(u, h, t);
  accumulate<float, MU, FWD>(acc, t);
}

// Persistent FP32 multi-RHS hop over tile records.  A block of MT_S x nr threads (site x RHS)
// loops over tiles blockIdx.x, + gridDim.x, ...; thread 0 stages the next tile's record into the
// other of two shared-memory buffers with one bulk copy while the block computes the current
// tile, so the record's latency hides behind the work.  A wait that does not end within MT_WAIT
// polls sets *err; the block then stops after its current tile and waits (bounded) for its
// copies in flight.
template <int EPI, bool G5>
__global__ void __launch_bounds__(MT_S* MR_MAXR, 2)
    k_hop_mrhs_t(Geom g, int nr, MrList lst, const float4* __restrict__ in, const float4* __restrict__ same,
                 float4* __restrict__ out, i64 rs, const unsigned char* __restrict__ rec0, int ntiles, float coef,
                 int* err) {
  constexpr bool NEEDC = EPI != EPI_HOP && EPI != EPI_XPAY;
  constexpr bool CI = EPI == EPI_INV || EPI == EPI_INVXPAY;
  // staged part of a record: its offset in the record, its size, and where each piece lands
  constexpr uint32_t SRC = (NEEDC && !CI) ? 0u : MT_OFF_NB;
  constexpr uint32_t BYTES = NEEDC ? MT_CLOV + MT_NB + MT_W : MT_NB + MT_W;
  constexpr uint32_t S_NB = (NEEDC && !CI) ? MT_CLOV : 0u, S_W = S_NB + MT_NB, S_CL = CI ? MT_NB + MT_W : 0u;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = (uint64_t*)(smem + 2 * BYTES);
  volatile int* failed = (volatile int*)(bar + 2);
  const int s = threadIdx.x, r = threadIdx.y, tid = r * MT_S + s;
  const i64 sv = g.sv;
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    *failed = 0;
    tc::fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int tile, int b) {
    tc::mbar_expect_tx(&bar[b], BYTES);
    tc::bulk_g2s(smem + b * BYTES, rec0 + (i64)tile * MT_REC + SRC, BYTES, &bar[b]);
  };
  if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  int i = 0;
  bool pending_next = false;  // a copy into the other buffer is in flight (thread 0's view)
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
    const int b = i & 1;
    pending_next = tile + (int)gridDim.x < ntiles;
    if (tid == 0 && pending_next) issue(tile + gridDim.x, b ^ 1);
    const bool ok = !*failed && tc::mbar_wait(&bar[b], (uint32_t)(i >> 1) & 1u, MT_WAIT);
    if (!ok) *failed = 1;
    const uint32_t cb = (uint32_t)tile * MT_S + s;
    if (ok && r < nr && cb < (uint32_t)g.Vh) {
      const unsigned char* buf = smem + b * BYTES;
      const uint32_t* nbt = (const uint32_t*)(buf + S_NB);
      const float2* wt = (const float2*)(buf + S_W);
      const float4* ct = (const float4*)(buf + S_CL);
      const i64 ro = (i64)lst.idx[r] * rs;
      const float4* inr = in + ro;
      cplx<float> acc[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = mk(0.f, 0.f);
      constexpr bool G5IN = G5 && EPI == EPI_INV;
      mt_leg<0, G5IN>(nbt, wt, s, inr, sv, acc);
      mt_leg<1, G5IN>(nbt, wt, s, inr, sv, acc);
      mt_leg<2, G5IN>(nbt, wt, s, inr, sv, acc);
      mt_leg<3, G5IN>(nbt, wt, s, inr, sv, acc);
      mt_leg<4, G5IN>(nbt, wt, s, inr, sv, acc);
      mt_leg<5, G5IN>(nbt, wt, s, inr, sv, acc);
      mt_leg<6, G5IN>(nbt, wt, s, inr, sv, acc);
      mt_leg<7, G5IN>(nbt, wt, s, inr, sv, acc);
      auto load = [&](const float4* f, cplx<float> v[12]) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          float4 q = __ldg(f + ro + j * sv + cb);
          v[2 * j] = mk(q.x, q.y);
          v[2 * j + 1] = mk(q.z, q.w);
        }
      };
      auto clover = [&](const cplx<float> v[12], cplx<float> y[12]) {
#pragma unroll
        for (int blk = 0; blk < 2; ++blk) {
          float c[36];
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const float4 q = ct[(blk * 9 + k) * MT_S + s];
            c[4 * k] = q.x;
            c[4 * k + 1] = q.y;
            c[4 * k + 2] = q.z;
            c[4 * k + 3] = q.w;
          }
          herm6_apply<float>(c, v + 6 * blk, y + 6 * blk);
        }
      };
      cplx<float> o[12];
      if (EPI == EPI_HOP) {
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = coef * acc[k];
      } else if (EPI == EPI_DFULL || EPI == EPI_DHAT2) {
        cplx<float> v[12], y[12];
        load(same, v);
        clover(v, y);
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
        clover(acc, o);
      } else if (EPI == EPI_INVXPAY) {
        cplx<float> v[12];
        load(same, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = v[k] + coef * acc[k];
        clover(v, o);
      } else {  // EPI_XPAY
        cplx<float> v[12];
        load(same, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = v[k] + coef * acc[k];
      }
      float4* outr = out + ro;
#pragma unroll
      for (int j = 0; j < 6; ++j)
        outr[j * sv + cb] = make_float4(o[2 * j].re, o[2 * j].im, o[2 * j + 1].re, o[2 * j + 1].im);
    }
    __syncthreads();  // every thread is done with buffer b before the next iteration refills it
    if (*failed) break;
  }
  if (tid == 0 && *failed) {
    atomicExch(err, 1);
    // the copy into the other buffer issued in the last iteration may still be in flight
    if (pending_next) tc::mbar_wait(&bar[(i & 1) ^ 1], (uint32_t)((i + 1) >> 1) & 1u, MT_WAIT);
  }
}

// The tile records of both parities, rebuilt when the gauge field or clover term changed.
static qxd_status mr_tiles(qxd_lattice* lat, const unsigned char** rec, int** err) {
  const Geom& g = lat->g;
  const i64 nt = (g.Vh + MT_S - 1) / MT_S;
  void *p, *e;
  const void* before = lat->work[MW_TILES];
  qxd_status st = ensure_work(lat, MW_TILES, (size_t)2 * nt * MT_REC, &p);
  if (st != QXD_OK) return st;
  st = ensure_work(lat, MW_TILE_ERR, sizeof(int), &e);
  if (st != QXD_OK) return st;
  if (lat->mrt_epoch != lat->epoch || before != p) {
    QXD_CUDA(lat, cudaMemsetAsync(e, 0, sizeof(int), lat->stream));
    for (int par = 0; par < 2; ++par) {
      const i64 n = nt * MT_S;
      k_mr_tiles<<<(unsigned)((n + 127) / 128), 128, 0, lat->stream>>>(g, par, lat->W32, lat->C32, lat->Ci32,
                                                                      (unsigned char*)p + (i64)par * nt * MT_REC, nt);
      QXD_CHECK_LAUNCH(lat, "k_mr_tiles");
    }
    lat->mrt_epoch = lat->epoch;
  }
  *rec = (const unsigned char*)p;
  *err = (int*)e;
  return QXD_OK;
}

qxd_status mrhs_tile_status(qxd_lattice* lat) {
  if (!lat->work[MW_TILE_ERR]) return QXD_OK;
  int h = 0;
  QXD_CUDA(lat, cudaMemcpyAsync(&h, lat->work[MW_TILE_ERR], sizeof(int), cudaMemcpyDeviceToHost, lat->stream));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  if (h) return fail(lat, QXD_ETIMEOUT, "a bounded wait of the multi-RHS hop expired");
  return QXD_OK;
}

template <int EPI, bool G5>
static qxd_status launch_mrhs_t(qxd_lattice* lat, int par, const float4* in, const float4* same, float4* out,
                                float coef, int nr, const MrList& lst, i64 rs, const unsigned char* rec, int* err) {
  constexpr bool NEEDC = EPI != EPI_HOP && EPI != EPI_XPAY;
  constexpr uint32_t BYTES = NEEDC ? MT_CLOV + MT_NB + MT_W : MT_NB + MT_W;
  constexpr size_t SMEM = 2 * BYTES + 2 * sizeof(uint64_t) + 16;
  static int blocks_per_sm = 0, sms = 0;
  if (!blocks_per_sm) {
    int dev = 0;
    QXD_CUDA(lat, cudaGetDevice(&dev));
    QXD_CUDA(lat, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    QXD_CUDA(lat, cudaFuncSetAttribute((const void*)k_hop_mrhs_t<EPI, G5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM));
    int b = 0;
    QXD_CUDA(lat, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_hop_mrhs_t<EPI, G5>, MT_S * MR_MAXR, SMEM));
    blocks_per_sm = b < 1 ? 1 : b;
  }
  const Geom& g = lat->g;
  const int ntiles = (int)((g.Vh + MT_S - 1) / MT_S);
  const i64 want = (i64)blocks_per_sm * sms;
  const unsigned grid = (unsigned)(ntiles < want ? ntiles : want);
  k_hop_mrhs_t<EPI, G5><<<grid, dim3(MT_S, nr), SMEM, lat->stream>>>(g, nr, lst, in, same, out, rs,
                                                                      rec + (i64)par * ntiles * MT_REC, ntiles, coef,
                                                                      err);
  QXD_CHECK_LAUNCH(lat, "k_hop_mrhs_t");
  return QXD_OK;
}

qxd_status hop32_mrhs(qxd_lattice* lat, int par, int epi, int g5, const float4* in, const float4* same, float4* out,
                      float coef, int nrhs, i64 rs, const int* rhs) {
  const Geom& g = lat->g;
  const unsigned char* rec;
  int* err;
  qxd_status st = mr_tiles(lat, &rec, &err);
  if (st != QXD_OK) return st;
  for (int r0 = 0; r0 < nrhs; r0 += MR_MAXR) {
    const int nr = nrhs - r0 < MR_MAXR ? nrhs - r0 : MR_MAXR;
    MrList lst;
    for (int r = 0; r < MR_MAXR; ++r) lst.idx[r] = r < nr ? (rhs ? rhs[r0 + r] : r0 + r) : 0;
    // bytes: per site and RHS the spinors; links and clover once per site for the whole block
    double sp = 96.0 * (2 + ((epi == EPI_DFULL || epi == EPI_DHAT2 || epi == EPI_INVXPAY || epi == EPI_XPAY) ? 1 : 0));
    double once = 8 * 72.0 + ((epi != EPI_HOP && epi != EPI_XPAY) ? 288.0 : 0.0);
    prof_begin(lat, KSTAT_F32_MRHS, (sp * nr + once) * (double)g.Vh);
#define QXD_MT_CASE(E, G) \
  if (epi == E && (g5 != 0) == G) st = launch_mrhs_t<E, G>(lat, par, in, same, out, coef, nr, lst, rs, rec, err); else
    QXD_MT_CASE(EPI_HOP, false)
    QXD_MT_CASE(EPI_DFULL, false)
    QXD_MT_CASE(EPI_INV, false)
    QXD_MT_CASE(EPI_INV, true)
    QXD_MT_CASE(EPI_DHAT2, false)
    QXD_MT_CASE(EPI_DHAT2, true)
    QXD_MT_CASE(EPI_XPAY, false)
    QXD_MT_CASE(EPI_INVXPAY, false) st = fail(lat, QXD_EINVAL, "unsupported multi-RHS epilogue");
#undef QXD_MT_CASE
    prof_end(lat);
    if (st != QXD_OK) return st;
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
      wl[i] = __ldg(W + link16_index(lp * 4 + mu, sv, k, fwd ? cb : sh.nbb[mu][ss]));
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
