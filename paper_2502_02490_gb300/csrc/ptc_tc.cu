// PTC layer with the channel mix on the 5th-generation tensor cores (tcgen05, BF16 in, FP32 out).
//
// For each output parity and colour a the layer is a real GEMM over a tile of 128 sites:
//   Out_a[x][n] = sum_k A_a[x][k] B[n][k],
//   k = (path p, input channel c', spin beta, re/im)   (K = 72 C_in),
//   n = (output channel c, spin alpha, re/im)           (N = 8 C_out, rounded up to 16),
// with A_a[x][(p, c', beta, r)] the real and imaginary parts of (T_p h_c')(x)[beta][a] (gauge
// transport of the input channel along path p) and B the 2x2 real form of the complex spin
// matrices Omega[c][c'][p][alpha][beta]:  [[Re, -Im], [Im, Re]].  Colour is a batch index that
// shares B, so the three colours are three MMAs into three TMEM column ranges.  K is cut into
// chunks of 64 = eight (path, channel) pairs of 8 reals, enumerated path-major.
//
// Persistent CTAs (one per SM) of 8 producer warps and 1 MMA warp walk the tiles.  A ring of
// TC_STAGES shared-memory stages holds the A chunks (and, when the layer's packed weights do not
// fit in shared memory, the B chunks, brought in by cp.async.bulk); "full" mbarriers tell the MMA
// warp that the producers (and the bulk copy) filled a stage, "empty" mbarriers (tcgen05.commit)
// tell the producers that the MMAs have read it.  Producers gauge-transport their (site, pair)
// items into the stage (FP32 links and spinors, rounded to BF16); one MMA thread issues 3 colours
// x 4 K-steps per chunk.  After a tile's last chunk the MMA thread commits to a "tile" mbarrier and
// the producers read their TMEM lanes (tcgen05.ld) and write the FP32 output channels, then go on
// to the next tile.  Every wait is bounded: on expiry the kernel sets the error word and stops;
// TMEM is freed on every exit path.
#include <cuda_bf16.h>

#include "qxd_internal.cuh"
#include "tc_common.cuh"

namespace qxd {

constexpr int TC_M = 128;          // sites per tile (MMA M)
constexpr int TC_KC = 64;          // K per chunk (8 pairs x 8 reals)
constexpr int TC_STAGES = 3;       // shared-memory ring
constexpr int TC_PROD = 512;       // producer threads (16 warps: 4 per site of the tile)
constexpr int TC_THREADS = TC_PROD + 32;
constexpr long long TC_WAIT = 1ll << 26;
constexpr uint32_t TC_ABYTES = 3u * TC_M * TC_KC * 2;  // one stage of A (three colours), 48 KB
constexpr size_t TC_SMEM_MAX = 200 * 1024;

struct TcLayer {
  Geom g;
  int cin, cout, np, nchunks;  // np = 8 cout rounded up to 16; nchunks = ceil(npaths cin / 8)
  int npaths;                  // 9: transport then mix; 1: mix only (first stage of the pull form)
  const void* in;              // [cin][2][6][sv] float4 (FP32) or uint2 (BF16 activations)
  void* out;                   // [cout][2][6][sv] float4 (FP32) or uint2 (BF16 activations)
  const float2* W;             // FP32 hop links
  const uint32_t* Wb;          // the same links as BF16 pairs, grouped layout (link16_index)
  const unsigned char* Bp;     // packed weights: [nchunks][np x 64 BF16, K-major core-matrix layout]
  int ntiles, tiles_per_par;   // tiles over both parities
  uint32_t tcols;              // TMEM columns allocated (power of 2 >= 3 np)
  int b_resident;              // 1: all B chunks preloaded once; 0: streamed per chunk
  int* err;
};

static int tc_np(int cout) { return (8 * cout + 15) & ~15; }
static int tc_nchunks(int cin, int npaths) { return (npaths * cin + 7) / 8; }

// Form of a layer: the pull form (mix at the source, then transport the output channels) when it
// has fewer output than input channels and its 9 C_out virtual channels fit in TMEM.
static bool tc_pull(int cin, int cout) { return cout < cin && 3 * tc_np(9 * cout) <= 512; }

// Packed BF16 weights of one layer in the K-major no-swizzle layout, B[j][n][k], zero padded.
// Push form: chunk j holds pairs q = 8 j .. 8 j + 7 (q = p cin + c'), n = (c, alpha, re/im).
// Pull form: chunk j holds input channels c' = 8 j .. 8 j + 7, n = (p cout + c, alpha, re/im).
__global__ void k_ptc_pack_w(int cin, int cout, int np, int nchunks, int pull, const float2* __restrict__ Om,
                             __nv_bfloat16* __restrict__ Bp) {
  const int per = np * TC_KC;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nchunks * per; e += gridDim.x * blockDim.x) {
    const int j = e / per, n = (e % per) / TC_KC, k = e % TC_KC;
    const int q = 8 * j + (k >> 3);
    float v = 0.f;
    const bool in_range = pull ? (n < 72 * cout && q < cin) : (n < 8 * cout && q < 9 * cin);
    if (in_range) {
      const int vc = n >> 3;  // output channel (push) or virtual channel p cout + c (pull)
      const int p = pull ? vc / cout : q / cin, ci = pull ? q : q % cin;
      const int c = pull ? vc % cout : vc, al = (n & 7) >> 1, ro = n & 1;
      const int be = (k & 7) >> 1, ri = k & 1;
      const float2 w = Om[(((i64)c * cin + ci) * 9 + p) * 16 + 4 * al + be];
      v = ro == 0 ? (ri == 0 ? w.x : -w.y) : (ri == 0 ? w.y : w.x);
    }
    unsigned char* base = (unsigned char*)Bp + (i64)j * per * 2;
    *(__nv_bfloat16*)(base + ((n >> 3) * (TC_KC >> 3) * 128 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2)) =
        __float2bfloat16_rn(v);
  }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *(uint32_t*)&h;
}

template <int MODE>  // 0: zero, 1: identity (path 0), 2: forward u h, 3: backward u^+ h
__device__ __forceinline__ void put_transported_m(unsigned char* a0, int s, int slot, const cplx<float> u[9],
                                                  const float4 raw[6]) {
  // spinor component (beta, b) = complex index 3 beta + b; float4 j holds complex 2 j, 2 j + 1
  auto comp = [&](int idx) -> cplx<float> {
    const float4 q = raw[idx >> 1];
    return (idx & 1) ? mk(q.z, q.w) : mk(q.x, q.y);
  };
  // one colour at a time: four spin components, packed and stored at once (few live registers)
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cplx<float> t[4];
#pragma unroll
    for (int be = 0; be < 4; ++be) {
      if constexpr (MODE == 0) {
        t[be] = mk(0.f, 0.f);
      } else if constexpr (MODE == 1) {
        t[be] = comp(3 * be + a);
      } else {
        cplx<float> r = mk(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; ++b)
          r = MODE == 2 ? cmac(r, u[3 * a + b], comp(3 * be + b)) : cjmac(r, u[3 * b + a], comp(3 * be + b));
        t[be] = r;
      }
    }
    uint4 v;
    v.x = pack_bf16x2(t[0].re, t[0].im);
    v.y = pack_bf16x2(t[1].re, t[1].im);
    v.z = pack_bf16x2(t[2].re, t[2].im);
    v.w = pack_bf16x2(t[3].re, t[3].im);
    *(uint4*)(a0 + a * (TC_ABYTES / 3) + tc::kmajor_off(s, 8 * slot, TC_KC)) = v;
  }
}

// Activations between layers are BF16 (four values per uint2, the float4 layout halved): the
// MMA operands are BF16 anyway, and half the bytes per load lets a producer keep both of its
// channels' loads in flight.  The network's input and output fields stay FP32.
template <bool IN16>
struct ActRaw {
  typedef float4 T;
};
template <>
struct ActRaw<true> {
  typedef uint2 T;
};

template <bool IN16>
__device__ __forceinline__ void act_load(const void* base, i64 off, i64 sv, typename ActRaw<IN16>::T raw[6]) {
  const typename ActRaw<IN16>::T* p = (const typename ActRaw<IN16>::T*)base + off;
#pragma unroll
  for (int jj = 0; jj < 6; ++jj) raw[jj] = __ldg(p + jj * sv);
}

__device__ __forceinline__ float4 act_f4(const float4 v) { return v; }
__device__ __forceinline__ float4 act_f4(const uint2 v) {
  return make_float4(B16::lo(v.x), B16::hi(v.x), B16::lo(v.y), B16::hi(v.y));
}

// The transported spinor of one input channel at one site (link u already carries the time sign):
// forward path t = u h, backward path t = u^+ h, path 0 t = h, written as BF16 into the three
// colour tiles of the stage, k = 8 slot + 2 beta + re/im (one 16-byte core-matrix row each).
// Separate instantiations per case, so that each executes only its own arithmetic.
__device__ __forceinline__ void put_transported(unsigned char* a0, int s, int slot, int p, bool fwd,
                                                const cplx<float> u[9], const float4 raw[6], bool zero) {
  if (zero)
    put_transported_m<0>(a0, s, slot, u, raw);
  else if (p == 0)
    put_transported_m<1>(a0, s, slot, u, raw);
  else if (fwd)
    put_transported_m<2>(a0, s, slot, u, raw);
  else
    put_transported_m<3>(a0, s, slot, u, raw);
}

// Checkerboard index of x + dir mu^ for a direction mu known only at run time (the path of a
// chunk), with `crossed` set on a wrap in direction mu: the map of nbr_cb32 (C* shift included),
// written with compile-time array indices only so that the coordinates stay in registers.
__host__ __device__ __forceinline__ uint32_t nbr_path32(const Geom& g, const int x[4], int mu, int dir,
                                                        bool& crossed) {
  int y[4];
  int v = 0, Lm = 1;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    y[k] = x[k];
    if (k == mu) {
      v = x[k];
      Lm = g.L[k];
    }
  }
  v += dir;
  crossed = v >= Lm || v < 0;
  v = v >= Lm ? 0 : (v < 0 ? Lm - 1 : v);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (k == mu) y[k] = v;
  if (crossed && g.shift && mu >= 2) {
    y[1] += g.shift;
    if (y[1] >= g.L[1]) y[1] -= g.L[1];
  }
  return ((((uint32_t)y[0] * g.L[1] + y[1]) * g.L[2] + y[2]) * g.L[3] + y[3]) >> 1;
}

// neighbour of site cb along path p (its checkerboard index and parity), and the path's link with
// the antiperiodic time sign folded in
__device__ __forceinline__ void path_setup(const TcLayer& L, int p, int par, uint32_t cb, const int x[4],
                                           uint32_t& src, int& spar, cplx<float> u[9]) {
  const Geom& g = L.g;
  src = cb;
  spar = par;
  if (p == 0) return;
  const bool fwd = p < 5;
  const int mu = fwd ? p - 1 : p - 5;
  bool cr;
  src = nbr_path32(g, x, mu, fwd ? +1 : -1, cr);
  spar = 1 - par;
  const float sign = (mu == 0 && cr && g.anti) ? -1.f : 1.f;
  const int lpar = fwd ? par : 1 - par;
  const uint32_t ls = fwd ? cb : src;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float2 w = __ldg(L.W + ((i64)(lpar * 4 + mu) * 9 + k) * g.sv + ls);
    u[k] = mk(sign * w.x, sign * w.y);
  }
}

#ifndef QXD_PTC_HMATH
#define QXD_PTC_HMATH 1  // BF16 activations: gauge transport in packed BF16 arithmetic
#endif

// Path 0 (MODE 1: the stored words as they are) or a site past the end of the lattice (MODE 0:
// zeros) for one BF16 input channel, written into the stage as the MMA operand
// (k = 8 slot + 2 beta + re/im).
template <int MODE>
__device__ __forceinline__ void put_plain_b16(unsigned char* a0, int s, int slot, const uint2 raw[6]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    uint32_t w[4];
#pragma unroll
    for (int be = 0; be < 4; ++be) {
      const int idx = 3 * be + a;  // complex component 3 beta + colour
      w[be] = MODE == 0 ? 0u : ((idx & 1) ? raw[idx >> 1].y : raw[idx >> 1].x);
    }
    *(uint4*)(a0 + a * (TC_ABYTES / 3) + tc::kmajor_off(s, 8 * slot, TC_KC)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// The raw operands of one chunk for one producer thread of a BF16 layer (C_in a multiple of 8):
// the path's link as BF16 words from the links' BF16 copy (grouped layout, three loads), the
// antiperiodic time sign as a flip of both halves' sign bits, and the two input channels' words.
struct ChunkRaw {
  uint32_t lw[9];
  uint2 r[2][6];
  int p;
  uint32_t sgn;
};

__device__ __forceinline__ void chunk_load(const TcLayer& L, int p, int cg8, int grp, bool live, int par,
                                           uint32_t cb, const int x[4], i64 cs, ChunkRaw& c) {
  const Geom& g = L.g;
  const int c0 = cg8 + 2 * grp;
  c.p = p;
  c.sgn = 0u;
  if (!live) {  // a site past the end of the lattice: zero operands (transported as zeros anyway)
#pragma unroll
    for (int k = 0; k < 9; ++k) c.lw[k] = 0u;
#pragma unroll
    for (int k = 0; k < 6; ++k) c.r[0][k] = c.r[1][k] = make_uint2(0u, 0u);
    return;
  }
  uint32_t src = cb;
  int spar = par;
  if (p == 0) {
#pragma unroll
    for (int k = 0; k < 9; ++k) c.lw[k] = 0u;  // the identity path uses no link
  } else {
    const bool fwd = p < 5;
    const int mu = fwd ? p - 1 : p - 5;
    bool cr;
    src = nbr_path32(g, x, mu, fwd ? +1 : -1, cr);
    spar = 1 - par;
    if (mu == 0 && cr && g.anti) c.sgn = 0x80008000u;
    const int lpar = fwd ? par : 1 - par;
    const uint32_t ls = fwd ? cb : src;
    const uint32_t* b = L.Wb + (i64)((lpar * 4 + mu) * 9) * g.sv;
    const uint4 w0 = __ldg((const uint4*)b + ls), w1 = __ldg((const uint4*)(b + 4 * g.sv) + ls);
    c.lw[0] = w0.x;
    c.lw[1] = w0.y;
    c.lw[2] = w0.z;
    c.lw[3] = w0.w;
    c.lw[4] = w1.x;
    c.lw[5] = w1.y;
    c.lw[6] = w1.z;
    c.lw[7] = w1.w;
    c.lw[8] = __ldg(b + 8 * g.sv + ls);
  }
  const i64 off = (i64)c0 * cs + (i64)spar * 6 * g.sv + src;
  act_load<true>(L.in, off, g.sv, c.r[0]);
  act_load<true>(L.in, off + cs, g.sv, c.r[1]);
}

// Gauge transport of one BF16 input channel in packed BF16 arithmetic, straight into the stage:
// the stored activation words (one complex number per 32-bit word, re low) times the link entries
// rounded to BF16, u x = (Re u, Re u) x + (-Im u, Im u) swap(x) (MODE 2, t = u h) and
// conj(u) x = (Re u, Re u) x + (Im u, -Im u) swap(x) (MODE 3, t = u^+ h) as packed fused
// multiply-adds.  ur and ui hold those link words, prepared once per chunk for both channels;
// each activation word is swapped once and feeds the three colour rows.  Each result word is
// already the BF16 operand the MMA reads (k = 8 slot + 2 beta + re/im).
template <int MODE>
__device__ __forceinline__ void transport_b16(unsigned char* a0, int s, int slot, const __nv_bfloat162 ur[9],
                                              const __nv_bfloat162 ui[9], const uint2 raw[6]) {
  __nv_bfloat162 t[3][4];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
#pragma unroll
    for (int be = 0; be < 4; ++be) {
      const int idx = 3 * be + b;
      const uint32_t w = (idx & 1) ? raw[idx >> 1].y : raw[idx >> 1].x;
      __nv_bfloat162 x;
      memcpy(&x, &w, 4);
      const __nv_bfloat162 xs = __lowhigh2highlow(x);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int k = MODE == 2 ? 3 * a + b : 3 * b + a;
        t[a][be] = b == 0 ? __hmul2(ur[k], x) : __hfma2(ur[k], x, t[a][be]);
        t[a][be] = __hfma2(ui[k], xs, t[a][be]);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    uint4 v;
    memcpy(&v.x, &t[a][0], 4);
    memcpy(&v.y, &t[a][1], 4);
    memcpy(&v.z, &t[a][2], 4);
    memcpy(&v.w, &t[a][3], 4);
    *(uint4*)(a0 + a * (TC_ABYTES / 3) + tc::kmajor_off(s, 8 * slot, TC_KC)) = v;
  }
}

template <int MODE>
__device__ __forceinline__ void chunk_transport(unsigned char* a0, int s, int grp, const ChunkRaw& c) {
  const __nv_bfloat162 sg = MODE == 2 ? __floats2bfloat162_rn(-1.f, 1.f) : __floats2bfloat162_rn(1.f, -1.f);
  __nv_bfloat162 ur[9], ui[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const uint32_t w = c.lw[k] ^ c.sgn;
    __nv_bfloat162 u;
    memcpy(&u, &w, 4);
    ur[k] = __low2bfloat162(u);
    ui[k] = __hmul2(__high2bfloat162(u), sg);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) transport_b16<MODE>(a0, s, 2 * grp + i, ur, ui, c.r[i]);
}

__device__ __forceinline__ void chunk_put(unsigned char* a0, int s, int grp, bool live, const ChunkRaw& c) {
  if (!live) {
#pragma unroll
    for (int i = 0; i < 2; ++i) put_plain_b16<0>(a0, s, 2 * grp + i, c.r[i]);
  } else if (c.p == 0) {
#pragma unroll
    for (int i = 0; i < 2; ++i) put_plain_b16<1>(a0, s, 2 * grp + i, c.r[i]);
  } else if (c.p < 5) {
    chunk_transport<2>(a0, s, grp, c);
  } else {
    chunk_transport<3>(a0, s, grp, c);
  }
}

// C_in a multiple of 8: chunk j is path p = j / (C_in / 8) and input channels cg8 + 0..7 with
// cg8 = 8 (j % (C_in / 8)); thread (s, grp) transports channels cg8 + 2 grp + 0..1 of its site.
// (Seventeen warps per SM leave each thread 96 registers: four SM sub-partitions of 16K
// registers, five warps on one of them.)
template <bool IN16>
__device__ __forceinline__ void transport_chunk_path(const TcLayer& L, unsigned char* a0, int p, int cg8, int s,
                                                     int grp, bool live, int par, uint32_t cb, const int x[4],
                                                     i64 cs) {
  const int c0 = cg8 + 2 * grp;
  uint32_t src;
  int spar;
  cplx<float> u[9];
  if constexpr (IN16 && QXD_PTC_HMATH != 0) {
    ChunkRaw c;
    chunk_load(L, p, cg8, grp, live, par, cb, x, cs, c);
    chunk_put(a0, s, grp, live, c);
    return;
  }
  if (live) path_setup(L, p, par, cb, x, src, spar, u);
  const i64 off = (i64)c0 * cs + (i64)spar * 6 * L.g.sv + src;
  if constexpr (IN16) {
    // BF16 activations: both channels' loads in flight at once (12 registers each)
    uint2 raw16[2][6];
    if (live) {
      act_load<true>(L.in, off, L.g.sv, raw16[0]);
      act_load<true>(L.in, off + cs, L.g.sv, raw16[1]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      float4 raw[6];
#pragma unroll
      for (int jj = 0; jj < 6; ++jj) raw[jj] = live ? act_f4(raw16[i][jj]) : make_float4(0.f, 0.f, 0.f, 0.f);
      put_transported(a0, s, 2 * grp + i, p, p < 5, u, raw, !live);
    }
  } else {
    // FP32 input: one channel's six loads in flight at a time (register budget)
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      float4 raw[6];
      if (live) act_load<false>(L.in, off + i * cs, L.g.sv, raw);
      put_transported(a0, s, 2 * grp + i, p, p < 5, u, raw, !live);
    }
  }
}

// general C_in: chunk j holds the pairs q = 8 j .. 8 j + 7 (q = p C_in + c', path-major); thread
// (s, grp) transports pairs 8 j + 2 grp + 0..1 (zero beyond npaths C_in)
template <bool IN16>
__device__ __forceinline__ void transport_chunk_pairs(const TcLayer& L, unsigned char* a0, int j, int s, int grp,
                                                      bool live, int par, uint32_t cb, const int x[4], i64 cs) {
  int last_p = -1;
  uint32_t src = cb;
  int spar = par;
  cplx<float> u[9];
#pragma unroll 1
  for (int i = 0; i < 2; ++i) {
    const int q = 8 * j + 2 * grp + i;
    const bool ok = live && q < L.npaths * L.cin;
    const int p = ok ? q / L.cin : 0, ci = ok ? q % L.cin : 0;
    float4 raw[6];
    if (ok) {
      if (p != last_p) {
        path_setup(L, p, par, cb, x, src, spar, u);
        last_p = p;
      }
      typename ActRaw<IN16>::T r16[6];
      act_load<IN16>(L.in, (i64)ci * cs + (i64)spar * 6 * L.g.sv + src, L.g.sv, r16);
#pragma unroll
      for (int jj = 0; jj < 6; ++jj) raw[jj] = act_f4(r16[jj]);
    }
    put_transported(a0, s, 2 * grp + i, p, p < 5, u, raw, !ok);
  }
}

// FAST: C_in a multiple of 8 (one path per chunk); else the general pair enumeration.  IN16 /
// OUT16: BF16 input / output activations.
template <bool FAST, bool IN16, bool OUT16>
__global__ void __launch_bounds__(TC_THREADS, 1) k_ptc_layer_tc(TcLayer L) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], tile_bar, bload;
  __shared__ uint32_t tbase;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Geom& g = L.g;
  const uint32_t bchunk = (uint32_t)(L.np * TC_KC * 2);
  unsigned char* sA = smem;                           // [TC_STAGES][3][128 x 64]
  unsigned char* sB = smem + TC_STAGES * TC_ABYTES;   // resident: [nchunks]; streamed: [TC_STAGES]
  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      tc::mbar_init(&full[s], TC_PROD + (L.b_resident ? 0 : 1));
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&tile_bar, 1);
    tc::mbar_init(&bload, 1);
    failed = 0;
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (warp == 0) tc::tmem_alloc(&tbase, L.tcols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  if (L.b_resident && tid == 0) {
    tc::mbar_expect_tx(&bload, bchunk * (uint32_t)L.nchunks);
    for (int j = 0; j < L.nchunks; ++j) tc::bulk_g2s(sB + (size_t)j * bchunk, L.Bp + (size_t)j * bchunk, bchunk, &bload);
  }
  const i64 cs = 12 * g.sv;  // channel stride (float4)
  int my_tiles = 0;
  for (int tile = blockIdx.x; tile < L.ntiles; tile += gridDim.x) ++my_tiles;

  if (warp == TC_PROD / 32) {
    // ---------------- MMA warp (one thread issues) ----------------
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(TC_M, L.np);
      constexpr uint32_t sbo = (TC_KC >> 3) * 128u;
      bool ok = !L.b_resident || tc::mbar_wait(&bload, 0, TC_WAIT);
      for (int it = 0; it < my_tiles && ok; ++it) {
        for (int j = 0; j < L.nchunks && ok; ++j) {
          const uint32_t cg = (uint32_t)(it * L.nchunks + j), st = cg % TC_STAGES, use = cg / TC_STAGES;
          if (!tc::mbar_wait(&full[st], use & 1, TC_WAIT)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const unsigned char* a0 = sA + st * TC_ABYTES;
          const unsigned char* b0 = L.b_resident ? sB + (size_t)j * bchunk : sB + (size_t)st * bchunk;
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int ks = 0; ks < TC_KC / 16; ++ks) {
              const uint64_t ad = tc::smem_desc(tc::smem_u32(a0 + a * (TC_ABYTES / 3)) + ks * 256, 128, sbo);
              const uint64_t bd = tc::smem_desc(tc::smem_u32(b0) + ks * 256, 128, sbo);
              tc::mma_bf16(tmem + (uint32_t)(a * L.np), ad, bd, idesc, (j > 0 || ks > 0) ? 1 : 0);
            }
          tc::mma_commit(&empty[st]);
        }
        if (ok) tc::mma_commit(&tile_bar);
      }
      if (!ok) {
        atomicExch(L.err, 1);
        failed = 1;
      }
    }
  } else {
    // ---------------- producers + epilogue ----------------
    const int s = tid & (TC_M - 1), grp = tid >> 7;  // site in the tile; pairs 2 grp, 2 grp + 1 of a chunk
    int it = 0;
    for (int tile = blockIdx.x; tile < L.ntiles; tile += gridDim.x, ++it) {
      if (*(volatile int*)&failed) break;
      const int par = tile / L.tiles_per_par;
      const uint32_t cb0 = (uint32_t)(tile % L.tiles_per_par) * TC_M;
      const uint32_t cb = cb0 + s;
      const bool live = cb < (uint32_t)g.Vh;
      int x[4] = {0, 0, 0, 0};
      if (live) cb_coords32(g, cb, par, x);
      bool ok = true;
      [[maybe_unused]] int p = 0, jg = 0;  // FAST: chunk j = p (C_in / 8) + jg, counted, not divided
      for (int j = 0; j < L.nchunks; ++j) {
        const uint32_t cg = (uint32_t)(it * L.nchunks + j), st = cg % TC_STAGES, use = cg / TC_STAGES;
        if (use > 0 && !tc::mbar_wait(&empty[st], (use - 1) & 1, TC_WAIT)) {
          ok = false;
          break;
        }
        if (!L.b_resident && tid == 0) {
          tc::mbar_expect_tx(&full[st], bchunk);
          tc::bulk_g2s(sB + (size_t)st * bchunk, L.Bp + (size_t)j * bchunk, bchunk, &full[st]);
        }
        unsigned char* a0 = sA + st * TC_ABYTES;
        if constexpr (FAST) {
          transport_chunk_path<IN16>(L, a0, p, 8 * jg, s, grp, live, par, cb, x, cs);
          if (++jg == (L.cin >> 3)) {
            jg = 0;
            ++p;
          }
        } else {
          transport_chunk_pairs<IN16>(L, a0, j, s, grp, live, par, cb, x, cs);
        }
        tc::fence_async_smem();
        tc::mbar_arrive(&full[st]);
      }
      if (!ok || !tc::mbar_wait(&tile_bar, it & 1, TC_WAIT)) {
        if (lane == 0) atomicExch(L.err, 1);
        failed = 1;
        break;
      }
      tc::fence_after_sync();
      // epilogue: warp w reads TMEM lanes 32 (w % 4) ..; the four warps of a lane group split the
      // output channels
      {
        const int lg = warp & 3, hw = warp >> 2;
        const uint32_t ocb = cb0 + 32 * lg + lane;
        const bool olive = ocb < (uint32_t)g.Vh;
        const int co_lo = (L.cout * hw) / 4, co_hi = (L.cout * (hw + 1)) / 4;
        for (int c = co_lo; c < co_hi; ++c) {
          float v[3][8];
#pragma unroll
          for (int a = 0; a < 3; ++a)
            tc::tmem_ld8(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(a * L.np + c * 8), v[a]);
          if (olive) {
            // complex index 3 alpha + a; float4 (or uint2) jj holds complex 2 jj, 2 jj + 1
#pragma unroll
            for (int jj = 0; jj < 6; ++jj) {
              const int k0 = 2 * jj, k1 = 2 * jj + 1;
              const float a = v[k0 % 3][2 * (k0 / 3)], b = v[k0 % 3][2 * (k0 / 3) + 1];
              const float cc = v[k1 % 3][2 * (k1 / 3)], d = v[k1 % 3][2 * (k1 / 3) + 1];
              if constexpr (OUT16)
                ((uint2*)L.out)[c * cs + (i64)par * 6 * g.sv + jj * g.sv + ocb] = make_uint2(B16::pack(a, b), B16::pack(cc, d));
              else
                ((float4*)L.out)[c * cs + (i64)par * 6 * g.sv + jj * g.sv + ocb] = make_float4(a, b, cc, d);
            }
          }
        }
      }
      tc::fence_before_sync();
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, L.tcols);
}

// Second stage of the pull form: out_c(x) = G_{0,c}(x) + sum_{p=1..8} (T_p G_{p,c})(x), with
// G_{p,c} the virtual channel p cout + c of the mix-only stage.  One thread per (site, channel).
template <bool IN16, bool OUT16>
__global__ void __launch_bounds__(256) k_ptc_pull(Geom g, int cout, const void* __restrict__ G,
                                                 const float2* __restrict__ W, void* __restrict__ out) {
  const i64 cs = 12 * g.sv;
  const i64 n = (i64)2 * g.Vh * cout;
  for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < n; e += (i64)gridDim.x * blockDim.x) {
    const uint32_t cb = (uint32_t)(e % g.Vh);
    const int par = (int)((e / g.Vh) & 1), c = (int)(e / (2 * g.Vh));
    cplx<float> acc[12];
    {
      typename ActRaw<IN16>::T r[6];
      act_load<IN16>(G, (i64)c * cs + (i64)par * 6 * g.sv + cb, g.sv, r);
#pragma unroll
      for (int jj = 0; jj < 6; ++jj) {
        const float4 q = act_f4(r[jj]);
        acc[2 * jj] = mk(q.x, q.y);
        acc[2 * jj + 1] = mk(q.z, q.w);
      }
    }
    int x[4];
    cb_coords32(g, cb, par, x);
#pragma unroll 1
    for (int p = 1; p < 9; ++p) {
      const bool fwd = p < 5;
      const int mu = fwd ? p - 1 : p - 5;
      bool cr;
      const uint32_t src = nbr_path32(g, x, mu, fwd ? +1 : -1, cr);
      const float sign = (mu == 0 && cr && g.anti) ? -1.f : 1.f;
      const int lpar = fwd ? par : 1 - par;
      const uint32_t ls = fwd ? cb : src;
      cplx<float> u[9], sp[12];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const float2 w = __ldg(W + ((i64)(lpar * 4 + mu) * 9 + k) * g.sv + ls);
        u[k] = mk(sign * w.x, sign * w.y);
      }
      typename ActRaw<IN16>::T r[6];
      act_load<IN16>(G, (i64)(p * cout + c) * cs + (i64)(1 - par) * 6 * g.sv + src, g.sv, r);
#pragma unroll
      for (int jj = 0; jj < 6; ++jj) {
        const float4 q = act_f4(r[jj]);
        sp[2 * jj] = mk(q.x, q.y);
        sp[2 * jj + 1] = mk(q.z, q.w);
      }
      if (fwd) {  // separate loops: each path executes only its own products
#pragma unroll
        for (int be = 0; be < 4; ++be)
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) acc[3 * be + a] = cmac(acc[3 * be + a], u[3 * a + b], sp[3 * be + b]);
      } else {
#pragma unroll
        for (int be = 0; be < 4; ++be)
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) acc[3 * be + a] = cjmac(acc[3 * be + a], u[3 * b + a], sp[3 * be + b]);
      }
    }
    const i64 ob = (i64)c * cs + (i64)par * 6 * g.sv + cb;
#pragma unroll
    for (int jj = 0; jj < 6; ++jj) {
      if constexpr (OUT16)
        ((uint2*)out)[ob + jj * g.sv] =
            make_uint2(B16::pack(acc[2 * jj].re, acc[2 * jj].im), B16::pack(acc[2 * jj + 1].re, acc[2 * jj + 1].im));
      else
        ((float4*)out)[ob + jj * g.sv] =
            make_float4(acc[2 * jj].re, acc[2 * jj].im, acc[2 * jj + 1].re, acc[2 * jj + 1].im);
    }
  }
}

bool ptc_tc_pull(int cin, int cout) { return tc_pull(cin, cout); }

// packed weights of a layer (bytes), for the buffer size
size_t ptc_tc_packed_bytes(int cin, int cout) {
  if (tc_pull(cin, cout)) return (size_t)tc_nchunks(cin, 1) * tc_np(9 * cout) * TC_KC * 2;
  return (size_t)tc_nchunks(cin, 9) * tc_np(cout) * TC_KC * 2;
}

// scratch of the pull form (the 9 cout virtual channels), in float4
size_t ptc_tc_pull_scratch(int cin, int cout, i64 sv) { return tc_pull(cin, cout) ? (size_t)9 * cout * 12 * sv : 0; }

qxd_status ptc_pack_weights(qxd_lattice* lat, int cin, int cout, const float2* Om, void* Bp) {
  const bool pull = tc_pull(cin, cout);
  const int np = pull ? tc_np(9 * cout) : tc_np(cout), nch = tc_nchunks(cin, pull ? 1 : 9);
  const int n = nch * np * TC_KC;
  k_ptc_pack_w<<<(n + 255) / 256, 256, 0, lat->stream>>>(cin, cout, np, nch, pull ? 1 : 0, Om, (__nv_bfloat16*)Bp);
  QXD_CHECK_LAUNCH(lat, "k_ptc_pack_w");
  return QXD_OK;
}

static qxd_status launch_tc(qxd_lattice* lat, int cin, int cout, int npaths, const void* in, int in16, const void* Bp,
                            void* out, int out16, int* err);

// one layer: push form (transport then mix) or pull form (mix, then transport the outputs); the
// pull form's virtual channels are BF16 activations in `scratch`
qxd_status ptc_layer_tc(qxd_lattice* lat, int cin, int cout, const void* in, int in16, const void* Bp, void* out,
                        int out16, void* scratch, int* err) {
  if (!tc_pull(cin, cout)) return launch_tc(lat, cin, cout, 9, in, in16, Bp, out, out16, err);
  qxd_status st = launch_tc(lat, cin, 9 * cout, 1, in, in16, Bp, scratch, 1, err);
  if (st) return st;
  const i64 n = (i64)2 * lat->Vh * cout;
  const int grid = (int)std::min<i64>((n + 255) / 256, 152 * 16);
  prof_begin(lat, KSTAT_PTC_TC, (48.0 * 9 * cout + (out16 ? 48.0 : 96.0) * cout + 576.0) * (double)lat->V);
  if (out16)
    k_ptc_pull<true, true><<<grid, 256, 0, lat->stream>>>(lat->g, cout, scratch, lat->W32, out);
  else
    k_ptc_pull<true, false><<<grid, 256, 0, lat->stream>>>(lat->g, cout, scratch, lat->W32, out);
  prof_end(lat);
  QXD_CHECK_LAUNCH(lat, "k_ptc_pull");
  return QXD_OK;
}

template <bool FAST, bool IN16, bool OUT16>
static const void* tc_kernel() {
  return (const void*)k_ptc_layer_tc<FAST, IN16, OUT16>;
}

static qxd_status launch_tc(qxd_lattice* lat, int cin, int cout, int npaths, const void* in, int in16, const void* Bp,
                            void* out, int out16, int* err) {
  TcLayer L;
  L.g = lat->g;
  L.cin = cin;
  L.cout = cout;
  L.npaths = npaths;
  L.np = tc_np(cout);
  L.nchunks = tc_nchunks(cin, npaths);
  L.in = in;
  L.out = out;
  L.W = lat->W32;
  L.Wb = lat->WB16;
  L.Bp = (const unsigned char*)Bp;
  L.tiles_per_par = (int)((lat->Vh + TC_M - 1) / TC_M);
  L.ntiles = 2 * L.tiles_per_par;
  uint32_t cols = 32;
  while (cols < (uint32_t)(3 * L.np)) cols <<= 1;
  L.tcols = cols;
  L.err = err;
  const size_t bchunk = (size_t)L.np * TC_KC * 2;
  const size_t base = (size_t)TC_STAGES * TC_ABYTES;
  L.b_resident = base + bchunk * L.nchunks <= TC_SMEM_MAX;
  const size_t smem = base + bchunk * (L.b_resident ? L.nchunks : TC_STAGES);
  // the dynamic shared-memory limit is a per-device function attribute: set it for the kernel
  // about to run (a cheap host call, no synchronisation)
  const bool fast = cin % 8 == 0;
  const int variant = (fast ? 4 : 0) + (in16 ? 2 : 0) + (out16 ? 1 : 0);
  static const void* kernels[8] = {tc_kernel<false, false, false>(), tc_kernel<false, false, true>(),
                                   tc_kernel<false, true, false>(),  tc_kernel<false, true, true>(),
                                   tc_kernel<true, false, false>(),  tc_kernel<true, false, true>(),
                                   tc_kernel<true, true, false>(),   tc_kernel<true, true, true>()};
  QXD_CUDA(lat, cudaFuncSetAttribute(kernels[variant], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_MAX));
  int dev = 0, sms = 0;
  QXD_CUDA(lat, cudaGetDevice(&dev));
  QXD_CUDA(lat, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = L.ntiles < sms ? L.ntiles : sms;
  // algorithmic bytes: each input channel, the 8 links (when transporting) and each output channel
  // once per site
  prof_begin(lat, KSTAT_PTC_TC,
             ((in16 ? 48.0 : 96.0) * cin + (out16 ? 48.0 : 96.0) * cout + (npaths == 9 ? 576.0 : 0.0)) * (double)lat->V);
  void* args[] = {&L};
  const cudaError_t le = cudaLaunchKernel(kernels[variant], dim3(grid), dim3(TC_THREADS), args, smem, lat->stream);
  prof_end(lat);
  if (le != cudaSuccess) return cuda_fail(lat, le, "k_ptc_layer_tc");
  QXD_CHECK_LAUNCH(lat, "k_ptc_layer_tc");
  return QXD_OK;
}

}  // namespace qxd
