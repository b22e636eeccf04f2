// Schwarz alternating procedure (SAP) on the GPU, FP32: the preconditioner that the paper's CPU
// solves put inside GCR (Sec. 5.1, openQxD's DFL_SAP_GCR; the paper only names it).
//
// The lattice is cut into non-overlapping blocks of extents b_mu, with a block grid
// n_mu = L_mu / b_mu that is even in every direction (with C*, the mirror shift L1 is an even
// number of x blocks too).  So blocks of one colour (the parity of the block coordinates) never
// touch, and no block wraps around the lattice.
//
// One cycle sweeps colour 0 and then colour 1.  Each block of the colour runs nmr
// minimal-residual steps on its Dirichlet block operator D_Lambda (D with the hops that leave
// the block dropped) for the current residual, and adds the result to x.  Blocks of one colour
// are independent, so a sweep is one launch with one CTA per block, and the residual
// r = eta - D x is recomputed after the sweep.  That equals updating r block by block, because a
// block's correction changes r only on the block and on neighbouring blocks of the other colour.
//
// Kernel: one thread per block site (block volume <= 256).  The block residual lives in
// shared memory, where the neighbours' hops read it.  Links and the clover come from the FP32
// fields in global memory (L2-resident across the steps), and each step reduces <D r, r> and
// ||D r||^2 over the CTA: warp shuffles, then the warp partials in warp order.
#include "hop_common.cuh"
#include "sap.cuh"
#include "trace.cuh"

namespace qxd {

constexpr int SAP_MAXVB = 256;
#ifndef QXD_SAP_MINB
#define QXD_SAP_MINB 2  // resident CTAs of 256 threads per SM: caps the block kernel at 128 registers
#endif

struct SapGeom {
  int b[4];       // block extents
  int n[4];       // block grid
  int stride[4];  // local lexicographic strides inside a block (x3 fastest)
  int vb;         // block volume = threads per CTA
  int nblocks;    // blocks of both colours
};

static qxd_status sap_geometry(qxd_lattice* lat, const int b[4], SapGeom* sg) {
  const Geom& g = lat->g;
  sg->vb = 1;
  sg->nblocks = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (b[mu] < 1 || g.L[mu] % b[mu]) return fail(lat, QXD_EINVAL, "SAP block extents must divide the lattice");
    sg->b[mu] = b[mu];
    sg->n[mu] = g.L[mu] / b[mu];
    if (sg->n[mu] % 2) return fail(lat, QXD_EINVAL, "SAP needs an even number of blocks in every direction");
    sg->vb *= b[mu];
    sg->nblocks *= sg->n[mu];
  }
  // C*: a hop across the y or z boundary also moves x by the physical L1 (Sec. 4.2).  Blocks
  // that meet there keep opposite colours only if that shift is an even number of x blocks.
  if (g.shift && g.shift % (2 * b[1]))
    return fail(lat, QXD_EINVAL, "SAP with C*: the physical L1 must be an even number of x blocks");
  if (sg->vb > SAP_MAXVB) return fail(lat, QXD_EINVAL, "SAP block volume must be at most 256 sites");
  sg->stride[3] = 1;
  for (int mu = 2; mu >= 0; --mu) sg->stride[mu] = sg->stride[mu + 1] * b[mu + 1];
  return QXD_OK;
}

qxd_status sap_check(qxd_lattice* lat, const int b[4]) {
  SapGeom sg;
  return sap_geometry(lat, b, &sg);
}

// One hop leg of D_Lambda at the thread's site: the neighbour's residual from shared memory,
// nothing when the neighbour lies outside the block (Dirichlet).
template <int LEG>
__device__ __forceinline__ void sap_leg(const Geom& g, const SapGeom& sg, const float2* __restrict__ W,
                                        const float4* rr, int s, const int lc[4], const int xg[4], int par,
                                        cplx<float> acc[12]) {
  constexpr int MU = LEG >> 1;
  constexpr bool FWD = (LEG & 1) == 0;
  const int l2 = lc[MU] + (FWD ? 1 : -1);
  if (l2 < 0 || l2 >= sg.b[MU]) return;
  const int s2 = s + (FWD ? sg.stride[MU] : -sg.stride[MU]);
  cplx<float> v[12], h[6], u[9], t[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float4 q = rr[j * sg.vb + s2];
    v[2 * j] = mk(q.x, q.y);
    v[2 * j + 1] = mk(q.z, q.w);
  }
  project<float, MU, FWD>(v, h);
  // forward: W_mu(x) stored at x; backward: W_mu(x - mu) stored at the neighbour (other parity)
  int y[4] = {xg[0], xg[1], xg[2], xg[3]};
  if (!FWD) y[MU] -= 1;
  const i64 site = lexi(g, y) >> 1;
  const int lp = FWD ? par : 1 - par;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float2 w = __ldg(W + ((i64)(lp * 4 + MU) * 9 + k) * g.sv + site);
    u[k] = mk(w.x, w.y);
  }
  link_mul<float, !FWD>(u, h, t);
  accumulate<float, MU, FWD>(acc, t);
}

// nmr minimal-residual steps on every block of one colour: e = 0, rr = r on the block;
// each step: a = D_Lambda rr, alpha = <a, rr> / <a, a>, e += alpha rr, rr -= alpha a.
// Then x += e.  r and x are full FP32 fields (parity planes [2][6][sv]).
__global__ void __launch_bounds__(SAP_MAXVB, QXD_SAP_MINB) k_sap_block_mr(Geom g, SapGeom sg, int colour, int nmr,
                                                            const float4* __restrict__ r, float4* __restrict__ x,
                                                            const float2* __restrict__ W,
                                                            const float4* __restrict__ C) {
  extern __shared__ float4 sap_sm[];
  float4* rr = sap_sm;                            // [6][vb] block residual
  float* part = (float*)(sap_sm + 6 * sg.vb);     // [3][SAP_MAXVB] per-thread partial sums
  float* alpha_sm = part + 3 * SAP_MAXVB;         // [2] the step length
  int kb[4], t = blockIdx.x;
  for (int mu = 3; mu >= 0; --mu) {
    kb[mu] = t % sg.n[mu];
    t /= sg.n[mu];
  }
  if (((kb[0] + kb[1] + kb[2] + kb[3]) & 1) != colour) return;  // the whole CTA: no barrier reached
  // the CTA is rounded up to whole warps (the shuffle reduction needs full warps): threads beyond
  // the block volume compute on site 0, add nothing and store nothing
  const bool act = (int)threadIdx.x < sg.vb;
  const int s = act ? (int)threadIdx.x : 0;
  int lc[4], xg[4], u = s;
  for (int mu = 3; mu >= 0; --mu) {
    lc[mu] = u % sg.b[mu];
    u /= sg.b[mu];
  }
  for (int mu = 0; mu < 4; ++mu) xg[mu] = kb[mu] * sg.b[mu] + lc[mu];
  const int par = (xg[0] + xg[1] + xg[2] + xg[3]) & 1;
  const i64 cb = lexi(g, xg) >> 1;
  const i64 base = (i64)par * 6 * g.sv + cb;
  // this site's residual lives only in shared memory (rr), where the neighbours read it too
  auto my_rr = [&](cplx<float> v[12]) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float4 q = rr[j * sg.vb + s];
      v[2 * j] = mk(q.x, q.y);
      v[2 * j + 1] = mk(q.z, q.w);
    }
  };
  cplx<float> e[12];
  if (act)
#pragma unroll
    for (int j = 0; j < 6; ++j) rr[j * sg.vb + s] = __ldg(r + base + (i64)j * g.sv);
#pragma unroll
  for (int k = 0; k < 12; ++k) e[k] = mk(0.f, 0.f);
  __syncthreads();
  for (int it = 0; it < nmr; ++it) {
    // a = D_Lambda rr at this site: A rr - 1/2 (the hops inside the block), built in acc
    cplx<float> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = mk(0.f, 0.f);
    sap_leg<0>(g, sg, W, rr, s, lc, xg, par, acc);
    sap_leg<1>(g, sg, W, rr, s, lc, xg, par, acc);
    sap_leg<2>(g, sg, W, rr, s, lc, xg, par, acc);
    sap_leg<3>(g, sg, W, rr, s, lc, xg, par, acc);
    sap_leg<4>(g, sg, W, rr, s, lc, xg, par, acc);
    sap_leg<5>(g, sg, W, rr, s, lc, xg, par, acc);
    sap_leg<6>(g, sg, W, rr, s, lc, xg, par, acc);
    sap_leg<7>(g, sg, W, rr, s, lc, xg, par, acc);
    cplx<float> me[12];
    my_rr(me);
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
      float cl[36];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float4 c = __ldg(C + ((i64)(par * 2 + blk) * 9 + k) * g.sv + cb);
        cl[4 * k] = c.x;
        cl[4 * k + 1] = c.y;
        cl[4 * k + 2] = c.z;
        cl[4 * k + 3] = c.w;
      }
      cplx<float> y[6];
      herm6_apply<float>(cl, me + 6 * blk, y);
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[6 * blk + k] = y[k] + (-0.5f) * acc[6 * blk + k];
    }
    float p_re = 0.f, p_im = 0.f, p_nn = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const cplx<float> a = acc[k];
      // <a, rr> = sum conj(a) rr and ||a||^2
      p_re = fmaf(a.re, me[k].re, fmaf(a.im, me[k].im, p_re));
      p_im = fmaf(a.re, me[k].im, fmaf(-a.im, me[k].re, p_im));
      p_nn = fmaf(a.re, a.re, fmaf(a.im, a.im, p_nn));
    }
    // warp sums by shuffles, then thread 0 adds the warp partials in warp order (fixed order:
    // the same bits every run); two barriers per step
    if (!act) p_re = p_im = p_nn = 0.f;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (sg.vb + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      p_re += __shfl_xor_sync(0xffffffffu, p_re, o);
      p_im += __shfl_xor_sync(0xffffffffu, p_im, o);
      p_nn += __shfl_xor_sync(0xffffffffu, p_nn, o);
    }
    if (lane == 0) {
      part[wid] = p_re;
      part[SAP_MAXVB + wid] = p_im;
      part[2 * SAP_MAXVB + wid] = p_nn;
    }
    __syncthreads();  // also: every thread has finished reading rr for this step
    if (threadIdx.x == 0) {
      float sre = 0.f, sim = 0.f, nn = 0.f;
      for (int k = 0; k < nw; ++k) {
        sre += part[k];
        sim += part[SAP_MAXVB + k];
        nn += part[2 * SAP_MAXVB + k];
      }
      alpha_sm[0] = nn > 0.f ? sre / nn : 0.f;
      alpha_sm[1] = nn > 0.f ? sim / nn : 0.f;
    }
    __syncthreads();
    const cplx<float> alpha = mk(alpha_sm[0], alpha_sm[1]);
    my_rr(me);  // reloaded: fewer live registers across the reduction
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      e[k] = cmac(e[k], alpha, me[k]);
      me[k] = me[k] - cmul(alpha, acc[k]);
    }
    if (act)
#pragma unroll
      for (int j = 0; j < 6; ++j)
        rr[j * sg.vb + s] = make_float4(me[2 * j].re, me[2 * j].im, me[2 * j + 1].re, me[2 * j + 1].im);
    __syncthreads();  // the new residual is complete before the next step's hops read it
  }
  if (!act) return;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float4 q = x[base + (i64)j * g.sv];
    q.x += e[2 * j].re;
    q.y += e[2 * j].im;
    q.z += e[2 * j + 1].re;
    q.w += e[2 * j + 1].im;
    x[base + (i64)j * g.sv] = q;
  }
}

static size_t sap_smem(const SapGeom& sg) { return sizeof(float4) * 6 * sg.vb + sizeof(float) * (3 * SAP_MAXVB + 2); }

// z = M r: ncy SAP cycles from z = 0 on full FP32 fields (internal layout).  Scratch: work
// slots 41 (residual) and 42 (D z).
qxd_status sap32(qxd_lattice* lat, const int b[4], int ncy, int nmr, const float4* rin, float4* z) {
  SapGeom sg;
  qxd_status st;
  if ((st = sap_geometry(lat, b, &sg))) return st;
  if (ncy < 1 || nmr < 1) return fail(lat, QXD_EINVAL, "SAP cycles and MR steps must be >= 1");
  const i64 sv = lat->sv, n4 = 12 * sv;
  const size_t fb = sizeof(float4) * n4;
  float4 *rs, *dz;
  if ((st = ensure_work(lat, 41, fb, (void**)&rs))) return st;
  if ((st = ensure_work(lat, 42, fb, (void**)&dz))) return st;
  if ((st = blas_zero(lat, z, fb))) return st;
  const size_t smem = sap_smem(sg);
  QXD_CUDA(lat, cudaFuncSetAttribute((const void*)k_sap_block_mr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  const float4* rcur = rin;
  for (int cy = 0; cy < ncy; ++cy) {
    for (int colour = 0; colour < 2; ++colour) {
      // algorithmic bytes of a sweep, per site of the colour: the residual read, x read and
      // written, 8 links and the clover pair once (the MR steps re-read them through L1/L2)
      prof_begin(lat, KSTAT_SAP, (3 * 96.0 + 8 * 72.0 + 288.0) * (double)lat->Vh);
      k_sap_block_mr<<<sg.nblocks, (sg.vb + 31) / 32 * 32, smem, lat->stream>>>(lat->g, sg, colour, nmr, rcur, z, lat->W32,
                                                                lat->C32);
      prof_end(lat);
      QXD_CHECK_LAUNCH(lat, "k_sap_block_mr");
      if (cy == ncy - 1 && colour == 1) break;  // the last sweep needs no new residual
      // r = rin - D z with the full FP32 operator
      if ((st = hop32(lat, 0, EPI_DFULL, 0, z + 6 * sv, z, dz, 0.f))) return st;
      if ((st = hop32(lat, 1, EPI_DFULL, 0, z, z + 6 * sv, dz + 6 * sv, 0.f))) return st;
      if ((st = blas_copy(lat, rs, rin, fb))) return st;
      if ((st = blas_axpy_32(lat, -1.0f, dz, rs, n4))) return st;
      rcur = rs;
    }
  }
  return QXD_OK;
}

}  // namespace qxd

using namespace qxd;

extern "C" qxd_status qxd_sap_apply(qxd_lattice* lat, double* out, const double* in, const int block[4], int ncy,
                                    int nmr, int on_device) {
  QXD_TRACE();
  if (!lat) return QXD_EINVAL;
  if (!out || !in || !block) return fail(lat, QXD_EINVAL, "null argument");
  if (!lat->have_clover) return fail(lat, QXD_ESTATE, "SAP before build_clover");
  const i64 sv = lat->sv;
  const size_t vb = sizeof(double) * 24 * lat->V;
  double2 *f64, *g64;
  float4 *a32, *b32;
  void *bi = nullptr, *bo = nullptr;
  qxd_status st;
  if ((st = ensure_work(lat, 24, sizeof(double2) * 24 * sv, (void**)&f64))) return st;
  if ((st = ensure_work(lat, 25, sizeof(double2) * 24 * sv, (void**)&g64))) return st;
  if ((st = ensure_work(lat, 43, sizeof(float4) * 12 * sv, (void**)&a32))) return st;
  if ((st = ensure_work(lat, 44, sizeof(float4) * 12 * sv, (void**)&b32))) return st;
  const double* src = in;
  if (!on_device) {
    if ((st = ensure_work(lat, 26, vb, &bi))) return st;
    if ((st = ensure_work(lat, 27, vb, &bo))) return st;
    QXD_CUDA(lat, cudaMemcpyAsync(bi, in, vb, cudaMemcpyHostToDevice, lat->stream));
    src = (const double*)bi;
  }
  if ((st = pack_spinor64(lat, (const double2*)src, f64, 0))) return st;
  if ((st = f64_to_f32(lat, f64, a32, 12 * sv))) return st;
  if ((st = sap32(lat, block, ncy, nmr, a32, b32))) return st;
  if ((st = f32_to_f64(lat, b32, g64, 12 * sv))) return st;
  if ((st = unpack_spinor64(lat, g64, on_device ? (double2*)out : (double2*)bo, 0))) return st;
  if (!on_device) {
    QXD_CUDA(lat, cudaMemcpyAsync(out, bo, vb, cudaMemcpyDeviceToHost, lat->stream));
    QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  }
  return QXD_OK;
}
