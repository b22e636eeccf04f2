// Batched persistent solve: several independent lattices of uneven volume in one launch.
//
// qxd_solve_batch runs the mixed-precision scheme for n lattices at once.  Outer: per lattice the
// FP64 defect correction (r = b - D x in FP64, Schur source and reconstruction in FP32).  Inner:
// ONE cooperative persistent kernel runs FP32 BiCGStab on Dhat for all lattices together.  Its
// work list is the tiles (256 threads x sites-per-thread sites of one parity half) of every
// lattice; each phase sweeps the tiles of the lattices still iterating, and phases are separated
// by a grid barrier (seven per iteration).  Dot products are fused into the phase that produces
// their operands and leave one partial per tile; after the barrier every block sums the partials
// of every lattice itself (one warp per lattice, fixed order), so all blocks hold identical
// scalars and take identical decisions (convergence, breakdown) without further barriers.  The
// sums do not depend on the grid, so results are reproducible.  A lattice whose residual meets
// its target, or whose BiCGStab coefficients break down, freezes while the others iterate.
//
// Every barrier wait is bounded: on timeout the waiting block sets the error word, every block
// leaves at its next barrier, and the host reports QXD_ETIMEOUT (nothing hangs).
//
// The cooperative launch is captured once into a CUDA graph and the graph is replayed in every
// outer round and later call on the same lattice set (a direct launch is used where capture is
// refused); the host reads the lattices' residual norms between rounds.  The sites per thread are
// picked by a small autotuner that times each candidate once per set of volumes.
#include <chrono>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "hop_site.cuh"
#include "reduce.cuh"
#include "trace.cuh"

namespace qxd {

constexpr int BMAX = 16;      // lattices per batch
constexpr int BNV = 3;        // values per tile partial
constexpr int BTHREADS = 256; // threads per block
// Algorithmic bytes per parity-half site of the persistent kernel (FP32 fields of 96 B):
// setup reads bh and writes x y r rh p (576 B), the close x = y + x 288 B; a reliable update
// y += x, x = 0 (384 B), Dhat y with r = r_hat = p = bh - Dhat y (1056 + 1152 + 96 + 288 B); each BiCGStab iteration runs two Dhat (each: the INV
// hop 1056 B = 8 neighbours + out + 8 links of 72 B + clover 288 B; the DHAT2 hop 1152 B with its
// diagonal input) and the vector phases <rh,v> 96 (v is the hop's output), s 288, <t,s>,<t,t> 96,
// x/r 672, p 384 B; 96 B more are counted for rh in <rh,v>.
constexpr double BATCH_SETUP_BYTES = 576.0 + 288.0;  // + the closing x = y + x
constexpr double BATCH_RELIABLE_BYTES = 384.0 + 1056.0 + 1152.0 + 96.0 + 288.0;
constexpr double BATCH_ITER_BYTES = 2 * (1056.0 + 1152.0) + 192.0 + 288.0 + 96.0 + 672.0 + 384.0;

struct BLat {
  Geom g;
  const float2* W;
  const float4* C;
  const float4* Ci;
  float4 *bh, *x, *r, *rh, *p, *v, *s, *t, *tmp, *y;  // single-parity FP32 fields [6][sv] (tmp: odd half)
  double target2;                                  // ||r||^2 target of the inner solve
  int t0, nt;                                      // first global tile, tiles of this lattice
};

// Launch controls that may change between replays of the captured launch (device memory).
struct BatchCtl {
  long long spin_limit;  // polls of a barrier wait before it gives up
  double delta;          // reliable-update threshold
  int maxiter;           // inner iteration cap of this launch
  int pad;
};

struct BatchArgs {
  const BLat* L;
  int nlat, ntiles, spt;
  double* part;          // [ntiles][BNV] tile partials of the current reduction
  unsigned int* bar;     // barrier arrival counter, zero at launch
  int* err;              // 0 ok, 1 barrier timeout
  int* iters;            // [nlat] inner iterations of this launch
  int* brk;              // [nlat] BiCGStab breakdowns of this launch (each one restarts)
  int* rels;             // [nlat] reliable updates of this launch
  const BatchCtl* ctl;
};

// Per-block copy of the lattices' BiCGStab state (identical in every block).
struct BlkState {
  double rho[BMAX][2], alpha[BMAX][2], omega[BMAX][2], beta[BMAX][2];
  double sum[BMAX][BNV];
  double rmax[BMAX];  // largest ||r|| since the last reliable update
  int active[BMAX];   // still iterating (not converged, not given up)
  int rel[BMAX];      // in a reliable update this iteration (drop: discard x)
  int drop[BMAX];
  int work[BMAX];     // lattices of the next sweeps
  int iters[BMAX], brk[BMAX], rels[BMAX];
  int act_t0[BMAX + 1];  // prefix of the tile counts of the work lattices (work-list compaction)
  unsigned int epoch;
  int ok, any, anyrel;
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier: barrier number e (counted per block) completes when the arrival counter reaches
// e * gridDim.x.  The wait is bounded; returns false (for every thread) when the batch is in error.
__device__ __forceinline__ bool gbar(const BatchArgs& a, BlkState& st) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int target = (st.epoch += 1) * gridDim.x;
    __threadfence();
    atomicAdd(a.bar, 1u);
    const long long lim = __ldcg(&a.ctl->spin_limit);
    long long it = 0;
    int ok = 1;
    while ((int)(ld_acquire(a.bar) - target) < 0) {
      if (*(volatile int*)a.err) {
        ok = 0;
        break;
      }
      if (++it > lim) {
        atomicExch(a.err, 1);
        ok = 0;
        break;
      }
      if (it > 32) __nanosleep(32);
    }
    __threadfence();
    st.ok = ok && *(volatile int*)a.err == 0;
  }
  __syncthreads();
  return st.ok != 0;
}

// Rebuild the compacted work list of the lattices in st.work (thread 0; the caller syncs).
__device__ __forceinline__ void compact(const BatchArgs& a, BlkState& st) {
  int n = 0;
  for (int k = 0; k < a.nlat; ++k) {
    st.act_t0[k] = n;
    if (st.work[k]) n += a.L[k].nt;
  }
  st.act_t0[a.nlat] = n;
}

// Data written by other blocks earlier in this kernel (spinor fields, tile partials) is read
// through L2 only (ld.global.cg): L1 and the read-only path are not coherent across blocks within
// a launch.  Links and clover never change during the kernel and keep the read-only path.
struct SpinorF32CG {
  typedef float real;
  struct Raw {
    float4 v[6];
  };
  float4* p;
  i64 sv;
  __device__ __forceinline__ Raw fetch(uint32_t cb) const {
    Raw r;
#pragma unroll
    for (int j = 0; j < 6; ++j) r.v[j] = __ldcg(p + j * sv + cb);
    return r;
  }
  __device__ __forceinline__ float decode(const Raw& r, cplx<float> s[12]) const {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      s[2 * j] = mk(r.v[j].x, r.v[j].y);
      s[2 * j + 1] = mk(r.v[j].z, r.v[j].w);
    }
    return 1.0f;
  }
  __device__ __forceinline__ void load(i64 cb, cplx<float> s[12]) const {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      float4 v = __ldcg(p + j * sv + cb);
      s[2 * j] = mk(v.x, v.y);
      s[2 * j + 1] = mk(v.z, v.w);
    }
  }
  template <typename T>
  __device__ __forceinline__ void store(i64 cb, const cplx<T> s[12]) const {
#pragma unroll
    for (int j = 0; j < 6; ++j)
      p[j * sv + cb] = make_float4((float)s[2 * j].re, (float)s[2 * j].im, (float)s[2 * j + 1].re,
                                   (float)s[2 * j + 1].im);
  }
};

#define LD(ptr) __ldcg(ptr)

__device__ __forceinline__ float4 cax(float ar, float ai, float4 x, float4 y) {  // y + a x
  return make_float4(y.x + ar * x.x - ai * x.y, y.y + ar * x.y + ai * x.x, y.z + ar * x.z - ai * x.w,
                     y.w + ar * x.w + ai * x.z);
}
__device__ __forceinline__ void cdot4(float4 a, float4 b, float& re, float& im) {  // += conj(a) b
  re += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
  im += a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
}
__device__ __forceinline__ void cdiv(const double a[2], const double b[2], double o[2]) {
  const double d = b[0] * b[0] + b[1] * b[1];
  o[0] = (a[0] * b[0] + a[1] * b[1]) / d;
  o[1] = (a[1] * b[0] - a[0] * b[1]) / d;
}
__device__ __forceinline__ bool finite2(const double z[2]) { return isfinite(z[0]) && isfinite(z[1]); }

// Sweep the tiles of the active lattices (the compacted list, spread over all blocks);
// f(k, L, cb, v) adds this site's contributions to the NV partials, which are block-reduced and
// stored per tile (NV = 0: no reduction).
template <int NV, class F>
__device__ __forceinline__ void sweep(const BatchArgs& a, const BlkState& st, F f) {
  const int nw = st.act_t0[a.nlat];
  for (int j = blockIdx.x; j < nw; j += gridDim.x) {
    int k = 0;
    while (j >= st.act_t0[k + 1]) ++k;
    const int tl = j - st.act_t0[k];  // tile within lattice k
    const BLat& L = a.L[k];
    const int t = L.t0 + tl;
    const uint32_t base = (uint32_t)tl * (uint32_t)(a.spt * BTHREADS);
    double v[NV > 0 ? NV : 1] = {};
    for (int q = 0; q < a.spt; ++q) {
      const uint32_t cb = base + q * BTHREADS + threadIdx.x;
      if (cb < (uint32_t)L.g.Vh) f(k, L, cb, v);
    }
    if constexpr (NV > 0) {
      block_sum<NV, BTHREADS>(v);
      if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) a.part[(i64)t * BNV + j] = v[j];
      }
    }
  }
}

// After a barrier: st.sum[k][0..NV) = the tile partials of each active lattice summed in tile
// order (warp w takes lattices w, w + 8, ...; fixed lane striding and shuffle tree).
template <int NV>
__device__ __forceinline__ void lat_sums(const BatchArgs& a, BlkState& st) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = w; k < a.nlat; k += BTHREADS / 32) {
    if (!st.work[k]) continue;
    const BLat& L = a.L[k];
    double s[NV] = {};
    for (int t = L.t0 + lane; t < L.t0 + L.nt; t += 32) {
#pragma unroll
      for (int j = 0; j < NV; ++j) s[j] += __ldcg(a.part + (i64)t * BNV + j);
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      s[j] = warp_sum(s[j]);
      if (lane == 0) st.sum[k][j] = s[j];
    }
  }
  __syncthreads();
}

// Dhat-part hop phase INV: tmp = A_oo^-1 H_oe src (odd output), src = p, s or y.
__device__ __forceinline__ void hop_inv(const BatchArgs& a, const BlkState& st, int which) {
  sweep<0>(a, st, [&](int, const BLat& L, uint32_t cb, double*) {
    SpinorF32CG si{which == 0 ? L.p : which == 1 ? L.s : L.y, L.g.sv}, so{L.tmp, L.g.sv};
    LinkF32 lk{L.W, L.g.sv};
    CloverF32 cl{L.Ci, L.g.sv};
    hop_site<float, SpinorF32CG, SpinorF32CG, SpinorF32CG, LinkF32, CloverF32, EPI_INV, false, 2>(
        L.g, 1, cb, si, si, so, lk, cl, 1.0f);
  });
}

// DHAT2 hop at one site: out = A_ee src - 1/4 H_eo tmp, the result also returned in o.
__device__ __forceinline__ void hop_dhat2(const BLat& L, uint32_t cb, float4* src, float4* out, cplx<float> o[12]) {
  SpinorF32CG si{L.tmp, L.g.sv}, ss{src, L.g.sv}, so{out, L.g.sv};
  LinkF32 lk{L.W, L.g.sv};
  CloverF32 cl{L.C, L.g.sv};
  hop_site<float, SpinorF32CG, SpinorF32CG, SpinorF32CG, LinkF32, CloverF32, EPI_DHAT2, false, 2>(
      L.g, 0, cb, si, ss, so, lk, cl, -0.25f, o);
}

__device__ __forceinline__ float4 o4(const cplx<float> o[12], int j) {
  return make_float4(o[2 * j].re, o[2 * j].im, o[2 * j + 1].re, o[2 * j + 1].im);
}

// Work mask of the next sweeps (thread 0; the caller syncs): 0 = iterating lattices, 1 = active
// lattices, 2 = lattices in a reliable update, 3 = all lattices.
__device__ __forceinline__ void set_work(const BatchArgs& a, BlkState& st, int mode) {
  for (int k = 0; k < a.nlat; ++k)
    st.work[k] = mode == 0 ? st.active[k] && !st.rel[k] : mode == 1 ? st.active[k] : mode == 2 ? st.rel[k] : 1;
  compact(a, st);
}

// MINB: resident blocks per SM the registers are capped for (1: no cap; 2: 128 registers).
template <int MINB>
__global__ void __launch_bounds__(BTHREADS, MINB) k_batch_bicg(BatchArgs a) {
  __shared__ BlkState st;
  if (threadIdx.x < BMAX) {
    const int k = threadIdx.x;
    st.active[k] = k < a.nlat;
    st.iters[k] = st.brk[k] = st.rel[k] = st.drop[k] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st.epoch = 0;
    st.ok = 1;
    set_work(a, st, 3);
  }
  __syncthreads();
  const int maxiter = __ldcg(&a.ctl->maxiter);
  const double delta = __ldcg(&a.ctl->delta);
  // setup: x = y = 0, r = r_hat = p = bh; partials ||bh||^2
  sweep<1>(a, st, [&](int, const BLat& L, uint32_t cb, double* v) {
    float n2 = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const i64 i = j * L.g.sv + cb;
      const float4 b = LD(L.bh + i);
      L.x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      L.y[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      L.r[i] = b;
      L.rh[i] = b;
      L.p[i] = b;
      n2 += b.x * b.x + b.y * b.y + b.z * b.z + b.w * b.w;
    }
    v[0] += n2;
  });
  if (!gbar(a, st)) return;
  lat_sums<1>(a, st);
  if (threadIdx.x < a.nlat) {
    const int k = threadIdx.x;
    st.rho[k][0] = st.sum[k][0];
    st.rho[k][1] = 0.0;
    st.rmax[k] = sqrt(st.sum[k][0]);
    st.active[k] = st.sum[k][0] > a.L[k].target2;
  }
  __syncthreads();
  if (threadIdx.x == 0) set_work(a, st, 0);
  __syncthreads();
  for (int it = 0;; ++it) {
    if (threadIdx.x == 0) {
      int any = 0;
      for (int k = 0; k < a.nlat; ++k) {
        any |= st.active[k];
        st.iters[k] += st.active[k] && it < maxiter;
      }
      st.any = any && it < maxiter;
    }
    __syncthreads();
    if (!st.any) break;
    // v = Dhat p, with the partials of <r_hat, v>
    hop_inv(a, st, 0);
    if (!gbar(a, st)) return;
    sweep<2>(a, st, [&](int, const BLat& L, uint32_t cb, double* acc) {
      cplx<float> o[12];
      hop_dhat2(L, cb, L.p, L.v, o);
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int j = 0; j < 6; ++j) cdot4(LD(L.rh + j * L.g.sv + cb), o4(o, j), re, im);
      acc[0] += re;
      acc[1] += im;
    });
    if (!gbar(a, st)) return;
    // alpha = rho / <r_hat, v> (a breakdown sends the lattice to a reliable update); s = r - alpha v
    lat_sums<2>(a, st);
    if (threadIdx.x < a.nlat && st.work[threadIdx.x]) {
      const int k = threadIdx.x;
      cdiv(st.rho[k], st.sum[k], st.alpha[k]);
      if (!finite2(st.alpha[k])) {
        st.rel[k] = 1;
        st.brk[k] += 1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) set_work(a, st, 0);
    __syncthreads();
    sweep<0>(a, st, [&](int k, const BLat& L, uint32_t cb, double*) {
      const float ar = (float)-st.alpha[k][0], ai = (float)-st.alpha[k][1];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const i64 i = j * L.g.sv + cb;
        L.s[i] = cax(ar, ai, LD(L.v + i), LD(L.r + i));
      }
    });
    if (!gbar(a, st)) return;
    // t = Dhat s, with the partials of <t, s> and <t, t>
    hop_inv(a, st, 1);
    if (!gbar(a, st)) return;
    sweep<3>(a, st, [&](int, const BLat& L, uint32_t cb, double* acc) {
      cplx<float> o[12];
      hop_dhat2(L, cb, L.s, L.t, o);
      float re = 0.f, im = 0.f, tt = 0.f;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const float4 tv = o4(o, j);
        cdot4(tv, LD(L.s + j * L.g.sv + cb), re, im);
        tt += tv.x * tv.x + tv.y * tv.y + tv.z * tv.z + tv.w * tv.w;
      }
      acc[0] += re;
      acc[1] += im;
      acc[2] += tt;
    });
    if (!gbar(a, st)) return;
    // omega = <t, s> / <t, t>; x += alpha p + omega s; r = s - omega t; partials <r_hat, r>, ||r||^2
    lat_sums<3>(a, st);
    if (threadIdx.x < a.nlat && st.work[threadIdx.x]) {
      const int k = threadIdx.x;
      const double tt = st.sum[k][2];
      st.omega[k][0] = st.sum[k][0] / tt;
      st.omega[k][1] = st.sum[k][1] / tt;
      if (!(tt > 0.0) || !finite2(st.omega[k])) {  // x and r stay as they were
        st.rel[k] = 1;
        st.brk[k] += 1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) set_work(a, st, 0);
    __syncthreads();
    sweep<3>(a, st, [&](int k, const BLat& L, uint32_t cb, double* acc) {
      const float wr = (float)st.omega[k][0], wi = (float)st.omega[k][1];
      const float alr = (float)st.alpha[k][0], ali = (float)st.alpha[k][1];
      float re = 0.f, im = 0.f, rn = 0.f;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const i64 i = j * L.g.sv + cb;
        const float4 sj = LD(L.s + i);
        L.x[i] = cax(wr, wi, sj, cax(alr, ali, LD(L.p + i), LD(L.x + i)));
        const float4 rj = cax(-wr, -wi, LD(L.t + i), sj);
        L.r[i] = rj;
        cdot4(LD(L.rh + i), rj, re, im);
        rn += rj.x * rj.x + rj.y * rj.y + rj.z * rj.z + rj.w * rj.w;
      }
      acc[0] += re;
      acc[1] += im;
      acc[2] += rn;
    });
    if (!gbar(a, st)) return;
    // rho' = <r_hat, r>, beta = (rho'/rho)(alpha/omega); a reliable update when ||r|| fell below
    // delta times its largest value since the last one, met the target, or the step broke down
    lat_sums<3>(a, st);
    if (threadIdx.x < a.nlat && st.work[threadIdx.x]) {
      const int k = threadIdx.x;
      const double rn2 = st.sum[k][2];
      if (!isfinite(rn2)) {  // overflow in the update: drop x
        st.rel[k] = 1;
        st.drop[k] = 1;
        st.brk[k] += 1;
      } else {
        const double rn = sqrt(rn2);
        if (rn > st.rmax[k]) st.rmax[k] = rn;
        double q1[2], q2[2];
        cdiv(st.sum[k], st.rho[k], q1);
        cdiv(st.alpha[k], st.omega[k], q2);
        st.beta[k][0] = q1[0] * q2[0] - q1[1] * q2[1];
        st.beta[k][1] = q1[0] * q2[1] + q1[1] * q2[0];
        st.rho[k][0] = st.sum[k][0];
        st.rho[k][1] = st.sum[k][1];
        if (rn < delta * st.rmax[k] || rn2 <= a.L[k].target2) {
          st.rel[k] = 1;
        } else if (!finite2(st.beta[k])) {
          st.rel[k] = 1;
          st.brk[k] += 1;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int anyrel = 0;
      for (int k = 0; k < a.nlat; ++k) anyrel |= st.rel[k];
      st.anyrel = anyrel;
      set_work(a, st, 1);
    }
    __syncthreads();
    // p = r + beta (p - omega v); lattices in a reliable update: y += x (unless dropped), x = 0
    sweep<0>(a, st, [&](int k, const BLat& L, uint32_t cb, double*) {
      if (st.rel[k]) {
        const bool keep = !st.drop[k];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const i64 i = j * L.g.sv + cb;
          if (keep) {
            const float4 xv = LD(L.x + i), yv = LD(L.y + i);
            L.y[i] = make_float4(yv.x + xv.x, yv.y + xv.y, yv.z + xv.z, yv.w + xv.w);
          }
          L.x[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
      }
      const float wr = (float)st.omega[k][0], wi = (float)st.omega[k][1];
      const float br = (float)st.beta[k][0], bi = (float)st.beta[k][1];
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const i64 i = j * L.g.sv + cb;
        const float4 q = cax(-wr, -wi, LD(L.v + i), LD(L.p + i));
        L.p[i] = cax(br, bi, q, LD(L.r + i));
      }
    });
    if (!gbar(a, st)) return;
    if (st.anyrel) {
      // reliable update: r = bh - Dhat y, r_hat = p = r, rho = ||r||^2
      if (threadIdx.x == 0) set_work(a, st, 2);
      __syncthreads();
      hop_inv(a, st, 2);
      if (!gbar(a, st)) return;
      sweep<1>(a, st, [&](int, const BLat& L, uint32_t cb, double* acc) {
        cplx<float> o[12];
        hop_dhat2(L, cb, L.y, L.v, o);
        float n2 = 0.f;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const i64 i = j * L.g.sv + cb;
          const float4 b = LD(L.bh + i), dv = o4(o, j);
          const float4 rj = make_float4(b.x - dv.x, b.y - dv.y, b.z - dv.z, b.w - dv.w);
          L.r[i] = rj;
          L.rh[i] = rj;
          L.p[i] = rj;
          n2 += rj.x * rj.x + rj.y * rj.y + rj.z * rj.z + rj.w * rj.w;
        }
        acc[0] += n2;
      });
      if (!gbar(a, st)) return;
      lat_sums<1>(a, st);
      if (threadIdx.x < a.nlat && st.rel[threadIdx.x]) {
        const int k = threadIdx.x;
        const double rn2 = st.sum[k][0];
        st.rho[k][0] = rn2;
        st.rho[k][1] = 0.0;
        st.rmax[k] = sqrt(rn2);
        if (!(rn2 > a.L[k].target2) || st.brk[k] > 10) st.active[k] = 0;  // converged, or given up
        st.rel[k] = 0;
        st.drop[k] = 0;
        st.rels[k] += 1;
      }
      __syncthreads();
      if (threadIdx.x == 0) set_work(a, st, 0);
      __syncthreads();
    }
  }
  // the inner solution: x = y + x on every lattice (read by the host after the launch)
  if (threadIdx.x == 0) set_work(a, st, 3);
  __syncthreads();
  sweep<0>(a, st, [&](int, const BLat& L, uint32_t cb, double*) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const i64 i = j * L.g.sv + cb;
      const float4 xv = LD(L.x + i), yv = LD(L.y + i);
      L.x[i] = make_float4(yv.x + xv.x, yv.y + xv.y, yv.z + xv.z, yv.w + xv.w);
    }
  });
  if (blockIdx.x == 0 && threadIdx.x < a.nlat) {
    a.iters[threadIdx.x] = st.iters[threadIdx.x];
    a.brk[threadIdx.x] = st.brk[threadIdx.x];
    a.rels[threadIdx.x] = st.rels[threadIdx.x];
  }
}

}  // namespace qxd

using namespace qxd;

#define TRY(x)                   \
  do {                           \
    qxd_status _s = (x);         \
    if (_s != QXD_OK) return _s; \
  } while (0)

namespace {

std::mutex g_tune_mutex;
std::map<std::string, std::pair<int, int>> g_tuned;  // volumes of a lattice set -> (blocks/SM, sites/thread)
int g_last_spt = 0, g_last_minb = 0;
bool g_last_graph = false;
long long g_spin_limit = 20000000;  // ~1.3 s of 64 ns sleeps: far above any phase of these lattices
std::string g_cache_path;           // tuning cache file ("" = none)

// Tuning cache file: one line per tuned set of volumes,
//   qxd-batch-tune 1 <GPU name, spaces as _> <SM count> <volumes "V0,V1,...,"> <blocks/SM> <sites/thread>
// read when a set is not yet tuned in this process, appended to after tuning.  The file only
// saves tuning time: unreadable files and malformed lines are ignored.
std::string gpu_tag() {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown 0";
  std::string name(prop.name);
  for (char& ch : name)
    if (ch == ' ' || ch == '\t') ch = '_';
  return name + " " + std::to_string(prop.multiProcessorCount);
}

bool cache_lookup(const std::string& key, int* minb, int* spt) {
  if (g_cache_path.empty()) return false;
  FILE* f = std::fopen(g_cache_path.c_str(), "r");
  if (!f) return false;
  const std::string tag = gpu_tag();
  char line[1024];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    std::istringstream is(line);
    std::string magic, ver, gpu, sms, vols;
    int mb = 0, sp = 0;
    if (!(is >> magic >> ver >> gpu >> sms >> vols >> mb >> sp)) continue;
    if (magic != "qxd-batch-tune" || ver != "1" || gpu + " " + sms != tag || vols != key) continue;
    if ((mb == 1 || mb == 2) && (sp == 1 || sp == 2 || sp == 4)) {  // the last valid line wins
      *minb = mb;
      *spt = sp;
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void cache_store(const std::string& key, int minb, int spt) {
  if (g_cache_path.empty()) return;
  FILE* f = std::fopen(g_cache_path.c_str(), "a");
  if (!f) return;
  std::fprintf(f, "qxd-batch-tune 1 %s %s %d %d\n", gpu_tag().c_str(), key.c_str(), minb, spt);
  std::fclose(f);
}

}  // namespace

namespace qxd {

qxd_status apply_D64(qxd_lattice* lat, const double2* in, double2* out);
qxd_status params_current(qxd_lattice* lat, const qxd_solve_params* p, qxd_solve_params* q);

// Device state of a batch, kept on the batch's first lattice between calls (freed with it or
// when a call brings another lattice set): fields, reduction and barrier words, the captured
// launch.  The lattice set is matched by the lattices' addresses and plane strides.
struct BatchCache {
  std::vector<const qxd_lattice*> lats;
  std::vector<i64> svs;
  BLat* dL = nullptr;
  double* part = nullptr;  // [tiles at one site per thread][BNV]
  unsigned int* bar = nullptr;
  int* err = nullptr;
  int* iters = nullptr;  // [BMAX] iterations, [BMAX] breakdowns, [BMAX] reliable updates
  BatchCtl* ctl = nullptr;
  BatchCtl* h_ctl = nullptr;
  int* h_out = nullptr;  // err, iters[BMAX], brk[BMAX], rels[BMAX]
  std::vector<float4*> buf;  // per lattice: 10 FP32 halves + the FP32 full residual
  std::vector<double2*> r64, t64;
  std::vector<BLat> hL;
  int grid_max[2] = {0, 0};  // co-resident blocks of the two kernel instances
  int grid = 0, spt = 0, minb = 1, ntiles = 0;
  cudaStream_t side = nullptr;  // capture stream (capture is refused on the legacy stream)
  cudaGraphExec_t gexec = nullptr;
  int g_spt = -1, g_ntiles = -1, g_minb = -1;  // shape the graph was captured with
  bool graph_refused = false;
};

static void cache_free(void* p) {
  BatchCache* c = (BatchCache*)p;
  if (!c) return;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->side) cudaStreamDestroy(c->side);
  for (void* q : {(void*)c->dL, (void*)c->part, (void*)c->bar, (void*)c->err, (void*)c->iters,
                  (void*)c->ctl})
    if (q) cudaFree(q);
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  if (c->h_out) cudaFreeHost(c->h_out);
  for (float4* q : c->buf) if (q) cudaFree(q);
  for (double2* q : c->r64) if (q) cudaFree(q);
  for (double2* q : c->t64) if (q) cudaFree(q);
  delete c;
}

static qxd_status cache_make(qxd_lattice* const* lats, int n, BatchCache** out) {
  qxd_lattice* l0 = lats[0];
  BatchCache* c = new BatchCache;
  c->lats.assign(lats, lats + n);
  c->hL.resize(n);
  c->buf.resize(n, nullptr);
  c->r64.resize(n, nullptr);
  c->t64.resize(n, nullptr);
  cudaError_t e = cudaSuccess;
#define CM(call)                  \
  if (e == cudaSuccess) {         \
    e = (call);                   \
  }
  for (int k = 0; k < n; ++k) {
    const i64 sv = lats[k]->sv;
    c->svs.push_back(sv);
    CM(cudaMalloc(&c->buf[k], sizeof(float4) * 6 * sv * 12));
    CM(cudaMalloc(&c->r64[k], sizeof(double2) * 24 * sv));
    CM(cudaMalloc(&c->t64[k], sizeof(double2) * 24 * sv));
    // zero once: the packs and kernels write real sites only, and the FP64 norms run over the
    // padded planes, so the padding must stay zero
    CM(cudaMemsetAsync(c->buf[k], 0, sizeof(float4) * 6 * sv * 12, l0->stream));
    CM(cudaMemsetAsync(c->r64[k], 0, sizeof(double2) * 24 * sv, l0->stream));
    CM(cudaMemsetAsync(c->t64[k], 0, sizeof(double2) * 24 * sv, l0->stream));
  }
  int dev = 0, sms = 0, per_sm = 0;
  CM(cudaGetDevice(&dev));
  CM(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CM(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_bicg<1>, BTHREADS, 0));
  c->grid_max[0] = sms * (per_sm < 1 ? per_sm : 1);
  int per_sm2 = 0;
  CM(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_batch_bicg<2>, BTHREADS, 0));
  c->grid_max[1] = sms * (per_sm2 < 2 ? per_sm2 : 2);
  i64 tiles1 = 0;
  for (int k = 0; k < n; ++k) tiles1 += (lats[k]->Vh + BTHREADS - 1) / BTHREADS;
  CM(cudaMalloc(&c->dL, sizeof(BLat) * n));
  CM(cudaMalloc(&c->bar, sizeof(unsigned int) * 2));
  CM(cudaMalloc(&c->err, sizeof(int)));
  CM(cudaMalloc(&c->iters, sizeof(int) * 3 * BMAX));
  CM(cudaMemsetAsync(c->iters, 0, sizeof(int) * 3 * BMAX, l0->stream));
  CM(cudaMalloc(&c->ctl, sizeof(BatchCtl)));
  CM(cudaMallocHost(&c->h_ctl, sizeof(BatchCtl)));
  CM(cudaMallocHost(&c->h_out, sizeof(int) * (1 + 3 * BMAX)));
  CM(cudaMalloc(&c->part, sizeof(double) * BNV * tiles1));
  CM(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
#undef CM
  if (e != cudaSuccess) {
    cache_free(c);
    return cuda_fail(l0, e, "allocation of the batch state");
  }
  if (per_sm < 1) {
    cache_free(c);
    return fail(l0, QXD_ECUDA, "the persistent batch kernel cannot be resident");
  }
  *out = c;
  return QXD_OK;
}

static const void* batch_kernel(int minb) {
  return minb == 2 ? (const void*)k_batch_bicg<2> : (const void*)k_batch_bicg<1>;
}

static void layout_tiles(BatchCache& c, int minb, int spt) {
  const int tile = BTHREADS * spt;
  int t0 = 0;
  for (size_t k = 0; k < c.hL.size(); ++k) {
    c.hL[k].t0 = t0;
    c.hL[k].nt = (int)((c.lats[k]->Vh + tile - 1) / tile);
    t0 += c.hL[k].nt;
  }
  c.ntiles = t0;
  c.spt = spt;
  c.minb = minb;
  const int gm = c.grid_max[minb - 1];
  c.grid = gm < t0 ? gm : t0;  // no more blocks than tiles: cheaper barriers
}

static BatchArgs batch_args(const BatchCache& c) {
  BatchArgs a;
  a.L = c.dL;
  a.nlat = (int)c.lats.size();
  a.ntiles = c.ntiles;
  a.spt = c.spt;
  a.part = c.part;
  a.bar = c.bar;
  a.err = c.err;
  a.iters = c.iters;
  a.brk = c.iters + BMAX;
  a.rels = c.iters + 2 * BMAX;
  a.ctl = c.ctl;
  return a;
}

// One launch of the persistent kernel on stream S: controls, barrier and error words reset
// first; from the captured graph when available (captured on the side stream once per shape).
static qxd_status run_persistent(qxd_lattice* l0, BatchCache& c, int maxiter, double delta, bool allow_graph,
                                 bool* used_graph) {
  cudaStream_t S = l0->stream;
  c.h_ctl->spin_limit = g_spin_limit;
  c.h_ctl->maxiter = maxiter;
  c.h_ctl->delta = delta;
  cudaError_t e = cudaMemcpyAsync(c.ctl, c.h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, S);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.bar, 0, sizeof(unsigned int) * 2, S);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.err, 0, sizeof(int), S);
  if (e != cudaSuccess) return cuda_fail(l0, e, "batch launch setup");
  BatchArgs a = batch_args(c);
  void* args[] = {&a};
  if (allow_graph && !c.graph_refused &&
      (c.g_spt != c.spt || c.g_ntiles != c.ntiles || c.g_minb != c.minb || !c.gexec)) {
    if (c.gexec) cudaGraphExecDestroy(c.gexec);
    c.gexec = nullptr;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c.side, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t le = cudaLaunchCooperativeKernel(batch_kernel(c.minb), dim3(c.grid), dim3(BTHREADS), args, 0, c.side);
      cudaError_t ee = cudaStreamEndCapture(c.side, &graph);
      if (le == cudaSuccess && ee == cudaSuccess && graph) {
        if (cudaGraphInstantiate(&c.gexec, graph, 0) != cudaSuccess) c.gexec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
    }
    if (!c.gexec) {
      c.graph_refused = true;  // capture of the cooperative launch refused: launch directly from now on
      cudaGetLastError();
    } else {
      c.g_spt = c.spt;
      c.g_ntiles = c.ntiles;
      c.g_minb = c.minb;
    }
  }
  if (allow_graph && c.gexec) {
    e = cudaGraphLaunch(c.gexec, S);
    if (e != cudaSuccess) return cuda_fail(l0, e, "cudaGraphLaunch(batch)");
    *used_graph = true;
  } else {
    e = cudaLaunchCooperativeKernel(batch_kernel(c.minb), dim3(c.grid), dim3(BTHREADS), args, 0, S);
    if (e != cudaSuccess) return cuda_fail(l0, e, "cudaLaunchCooperativeKernel(k_batch_bicg)");
  }
  l0->launches++;
  return QXD_OK;
}

static qxd_status read_outcome(qxd_lattice* l0, BatchCache& c, int n) {
  cudaStream_t S = l0->stream;
  cudaError_t e = cudaMemcpyAsync(c.h_out, c.err, sizeof(int), cudaMemcpyDeviceToHost, S);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c.h_out + 1, c.iters, sizeof(int) * 3 * BMAX, cudaMemcpyDeviceToHost, S);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S);
  if (e != cudaSuccess) return cuda_fail(l0, e, "batch outcome");
  if (c.h_out[0] == 1) return fail(l0, QXD_ETIMEOUT, "a grid barrier of the persistent batch kernel timed out");
  (void)n;
  return QXD_OK;
}

static qxd_status solve_batch_impl(qxd_lattice* const* lats, int n, double* const* x, const double* const* b,
                                   const qxd_solve_params* prm, qxd_solve_info* info) {
  qxd_lattice* l0 = lats[0];
  cudaStream_t S = l0->stream;
  auto t0 = std::chrono::steady_clock::now();
  // the cached device state of this lattice set, or a new one
  BatchCache* c = (BatchCache*)l0->batch;
  bool match = c && (int)c->lats.size() == n;
  for (int k = 0; match && k < n; ++k) match = c->lats[k] == lats[k] && c->svs[k] == lats[k]->sv;
  if (!match) {
    if (c) {
      cudaStreamSynchronize(S);
      cache_free(c);
      l0->batch = nullptr;
    }
    TRY(cache_make(lats, n, &c));
    l0->batch = c;
    l0->batch_release = cache_free;
  }
  // lattice views (operator pointers are re-read: the clover may have been rebuilt)
  for (int k = 0; k < n; ++k) {
    qxd_lattice* L = lats[k];
    const i64 sv = L->sv;
    float4* h = c->buf[k];
    BLat& bl = c->hL[k];
    bl.g = L->g;
    bl.W = L->W32;
    bl.C = L->C32;
    bl.Ci = L->Ci32;
    bl.bh = h;
    bl.x = h + 6 * sv;
    bl.r = h + 12 * sv;
    bl.rh = h + 18 * sv;
    bl.p = h + 24 * sv;
    bl.v = h + 30 * sv;
    bl.s = h + 36 * sv;
    bl.t = h + 42 * sv;
    bl.tmp = h + 48 * sv;  // odd half; h + 54 sv .. 66 sv: the FP32 full residual (two halves)
    bl.y = h + 66 * sv;
  }
  std::string key;
  for (int k = 0; k < n; ++k) key += std::to_string(lats[k]->V) + ",";
  int spt = 0, minb = 1;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      minb = it->second.first;
      spt = it->second.second;
    } else if (cache_lookup(key, &minb, &spt) && c->grid_max[minb - 1] >= 1) {
      g_tuned[key] = {minb, spt};
    } else {
      minb = 1;
      spt = 0;
    }
  }
  layout_tiles(*c, minb, spt ? spt : 1);
  // x_k = 0 (kept in r64), b_k in the internal layout (kept in t64)
  std::vector<double> bnorm(n), rel(n, 1.0), tgt(n);
  std::vector<char> done(n, 0);
  std::vector<int> its(n, 0), brk(n, 0), rels(n, 0);
  const double delta = prm->reliable_delta > 0.0 && prm->reliable_delta < 1.0 ? prm->reliable_delta : 0.1;
  for (int k = 0; k < n; ++k) {
    qxd_lattice* L = lats[k];
    const i64 nf = 24 * L->sv;
    TRY(pack_spinor64(L, (const double2*)b[k], c->t64[k], 0));
    TRY(blas_norm2_64(L, c->t64[k], nf, SC_TMP0));
    double v;
    TRY(read_scalars(L, SC_TMP0, 1, &v));
    bnorm[k] = std::sqrt(v);
    QXD_CUDA(L, cudaMemsetAsync(c->r64[k], 0, sizeof(double2) * nf, S));
    if (bnorm[k] == 0.0) {
      done[k] = 1;
      rel[k] = 0.0;
    }
  }
  int total = 0, outer = 0;
  const int max_outer = prm->max_outer > 0 ? prm->max_outer : 20;
  bool graph_used = false;
  for (; outer <= max_outer; ++outer) {
    // residuals res = D x - b (FP64) and their norms
    int nact = 0;
    for (int k = 0; k < n; ++k) {
      if (done[k]) continue;
      qxd_lattice* L = lats[k];
      const i64 nf = 24 * L->sv;
      double2* res;
      TRY(ensure_work(L, 24, sizeof(double2) * nf, (void**)&res));
      TRY(apply_D64(L, c->r64[k], res));
      TRY(blas_axpy_64(L, -1.0, 0.0, c->t64[k], res, nf));
      TRY(blas_norm2_64(L, res, nf, SC_TMP0));
      double v;
      TRY(read_scalars(L, SC_TMP0, 1, &v));
      rel[k] = std::sqrt(v) / bnorm[k];
      if (!std::isfinite(rel[k])) return fail(l0, QXD_ENOCONV, "non-finite residual in the batch");
      if (rel[k] <= prm->tol) {
        done[k] = 1;
        continue;
      }
      tgt[k] = std::max(prm->inner_tol * std::sqrt(v), 0.5 * prm->tol * bnorm[k]);
      ++nact;
    }
    if (nact == 0 || outer == max_outer || total >= prm->maxiter) break;
    // Schur sources bh = r_e + 1/2 H_eo A_oo^-1 r_o (FP32, r = b - D x); converged lattices get bh = 0
    for (int k = 0; k < n; ++k) {
      qxd_lattice* L = lats[k];
      BLat& bl = c->hL[k];
      const i64 sv = L->sv;
      bl.target2 = done[k] ? 1e300 : tgt[k] * tgt[k];
      if (done[k]) {
        QXD_CUDA(L, cudaMemsetAsync(bl.bh, 0, sizeof(float4) * 6 * sv, S));
        continue;
      }
      double2* res = (double2*)L->work[24];
      float4* r32 = bl.tmp + 6 * sv;
      TRY(f64_to_f32(L, res, r32, 12 * sv));
      TRY(blas_axpy_32(L, -2.0f, r32, r32, 12 * sv));
      TRY(clover_apply32(L, 1, 1, r32 + 6 * sv, bl.t));
      TRY(hop32(L, 0, EPI_XPAY, 0, bl.t, r32, bl.bh, 0.5f));
    }
    // the tile shape (blocks per SM, sites per thread): tuned once per set of volumes, each
    // candidate timed on the first inner solve (at most 2000 iterations)
    if (!spt) {
      float best = 1e30f;
      int best_spt = 1, best_minb = 1;
      cudaEvent_t e0, e1;
      QXD_CUDA(l0, cudaEventCreate(&e0));
      QXD_CUDA(l0, cudaEventCreate(&e1));
      qxd_status ts = QXD_OK;
      for (int cand : {0x11, 0x21, 0x12, 0x22, 0x14}) {
        const int cm = cand >> 4, cs = cand & 15;
        if (c->grid_max[cm - 1] < 1) continue;
        layout_tiles(*c, cm, cs);
        cudaError_t e = cudaMemcpyAsync(c->dL, c->hL.data(), sizeof(BLat) * n, cudaMemcpyHostToDevice, S);
        if (e == cudaSuccess) e = cudaEventRecord(e0, S);
        if (e != cudaSuccess) {
          ts = cuda_fail(l0, e, "batch tuning");
          break;
        }
        bool ug = false;
        ts = run_persistent(l0, *c, std::min(2000, prm->maxiter), delta, false, &ug);
        if (ts == QXD_OK && (e = cudaEventRecord(e1, S)) != cudaSuccess) ts = cuda_fail(l0, e, "batch tuning");
        if (ts == QXD_OK) ts = read_outcome(l0, *c, n);
        if (ts != QXD_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          best_spt = cs;
          best_minb = cm;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (ts != QXD_OK) return ts;
      spt = best_spt;
      minb = best_minb;
      layout_tiles(*c, minb, spt);
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tuned[key] = {minb, spt};
      cache_store(key, minb, spt);
    }
    QXD_CUDA(l0, cudaMemcpyAsync(c->dL, c->hL.data(), sizeof(BLat) * n, cudaMemcpyHostToDevice, S));
    // the inner solve of every lattice: one persistent launch
    prof_begin(l0, KSTAT_BATCH, 0.0);
    TRY(run_persistent(l0, *c, prm->maxiter - total, delta, true, &graph_used));
    prof_end(l0);
    TRY(read_outcome(l0, *c, n));
    int mx = 0;
    double bytes = 0.0;
    for (int k = 0; k < n; ++k) {
      const int ik = c->h_out[1 + k];
      mx = std::max(mx, ik);
      its[k] += ik;
      brk[k] += c->h_out[1 + BMAX + k];
      rels[k] += c->h_out[1 + 2 * BMAX + k];
      bytes += (BATCH_SETUP_BYTES + BATCH_ITER_BYTES * (double)ik +
                BATCH_RELIABLE_BYTES * (double)c->h_out[1 + 2 * BMAX + k]) * (double)lats[k]->Vh;
    }
    prof_set_last_bytes(l0, bytes);
    total += mx;
    // reconstruction: x_e += y, x_o += A_oo^-1 (r_o + 1/2 H_oe y)
    for (int k = 0; k < n; ++k) {
      if (done[k]) continue;
      qxd_lattice* L = lats[k];
      BLat& bl = c->hL[k];
      const i64 sv = L->sv;
      float4* r32 = bl.tmp + 6 * sv;
      TRY(hop32(L, 1, EPI_INVXPAY, 0, bl.x, r32 + 6 * sv, bl.t, 0.5f));
      TRY(blas_acc_f32_into_f64(L, bl.x, c->r64[k], 6 * sv));
      TRY(blas_acc_f32_into_f64(L, bl.t, c->r64[k] + 12 * sv, 6 * sv));
    }
  }
  bool ok = true;
  for (int k = 0; k < n; ++k) {
    TRY(unpack_spinor64(lats[k], c->r64[k], (double2*)x[k], 0));
    ok = ok && done[k];
  }
  QXD_CUDA(l0, cudaStreamSynchronize(S));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int k = 0; k < n && info; ++k) {
    info[k].iters_inner = its[k];
    info[k].iters_outer = outer;
    info[k].reliable_updates = rels[k];
    info[k].true_rel_res = rel[k];
    info[k].seconds = secs;
    info[k].status = done[k] ? QXD_OK : QXD_ENOCONV;
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_last_spt = c->spt;
    g_last_minb = c->minb;
    g_last_graph = graph_used;
  }
  if (!ok) return fail(l0, QXD_ENOCONV, "some lattice of the batch did not reach the tolerance");
  return QXD_OK;
}

}  // namespace qxd

extern "C" qxd_status qxd_solve_batch(qxd_lattice* const* lats, int n, double* const* x, const double* const* b,
                                      const qxd_solve_params* prm, qxd_solve_info* info) {
  QXD_TRACE();
  if (!lats || n <= 0 || n > BMAX || !x || !b || !prm) return QXD_EINVAL;
  qxd_lattice* l0 = lats[0];
  if (!l0) return QXD_EINVAL;
  if (info) std::memset(info, 0, sizeof(qxd_solve_info) * n);
  qxd_solve_params pv;
  if (qxd::params_current(l0, prm, &pv) != QXD_OK) return QXD_EINVAL;
  prm = &pv;
  if (prm->use_x0) return fail(l0, QXD_EINVAL, "use_x0 is supported by qxd_solve only");
  if (!prm->on_device) return fail(l0, QXD_EINVAL, "qxd_solve_batch takes device pointers (on_device = 1)");
  for (int k = 0; k < n; ++k) {
    if (!lats[k] || !x[k] || !b[k]) return fail(l0, QXD_EINVAL, "null lattice or field");
    if (!lats[k]->have_clover) return fail(l0, QXD_ESTATE, "solve before build_clover");
    if (lats[k]->stream != l0->stream) return fail(l0, QXD_EINVAL, "the batch's lattices must share one stream");
    for (int j = 0; j < k; ++j)
      if (lats[j] == lats[k]) return fail(l0, QXD_EINVAL, "a lattice appears twice in the batch");
  }
  qxd_status st = solve_batch_impl(lats, n, x, b, prm, info);
  if (st != QXD_OK && st != QXD_ENOCONV && l0->batch) {  // drop the device state after a failure
    cudaStreamSynchronize(l0->stream);
    cache_free(l0->batch);
    l0->batch = nullptr;
  }
  return st;
}

extern "C" qxd_status qxd_batch_last_config(int* threads, int* sites_per_thread, int* blocks_per_sm, int* graph) {
  if (!threads || !sites_per_thread || !blocks_per_sm || !graph) return QXD_EINVAL;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  *threads = BTHREADS;
  *sites_per_thread = g_last_spt;
  *blocks_per_sm = g_last_minb;
  *graph = g_last_graph ? 1 : 0;
  return QXD_OK;
}

extern "C" qxd_status qxd_batch_tune_cache(const char* path) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_cache_path = path ? path : "";
  return QXD_OK;
}

extern "C" qxd_status qxd_batch_set_spin_limit(long long limit) {
  if (limit < 1) return QXD_EINVAL;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_spin_limit = limit;
  return QXD_OK;
}
