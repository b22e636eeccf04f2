// Gauge-equivariant parallel-transport convolution (PTC) network: the learned preconditioner.
//
// Layer: out_c(x) = sum_{c'} sum_{p=0..8} Omega[c][c'][p] (T_p h_{c'})(x), with T_0 the identity,
// T_{1+mu} h(x) = W_mu(x) h(x+mu) and T_{5+mu} h(x) = W_mu(x-mu)^+ h(x-mu) (hop links, hop
// boundary signs, C* neighbours), Omega a complex 4x4 spin matrix per (c, c', p).  The net is a
// chain of such linear layers 1 -> C -> ... -> 1 and is trained on (b = D v, v) pairs to minimise
// sum_i ||M(b_i) - v_i||^2 with Adam.
//
// Device layout: activations are full-lattice FP32 fields, channel-major [C][2][6][sv] float4;
// weights FP32 complex [Cout][Cin][9][4][4] per layer, all layers concatenated.
//
// Kernels:
//  k_ptc_layer : a block covers 32 output sites (one parity) x Cout threads; per path the block
//                transports all input channels of its sites into shared memory, then every thread
//                mixes them into its output channel (4x4 spin matrix per input channel).  With the
//                adjoint weights Omega'[c'][c][swap p] = Omega[c][c'][p]^+ the same kernel applies the
//                layer's adjoint (backpropagation to the input).
//  k_ptc_wgrad : dL/dOmega*[c][c'][p] = sum_{x,a} g_c(x)[s,a] conj(T_p h_{c'}(x)[t,a]); blocks of a
//                fixed path accumulate over site tiles and write per-block partials; k_ptc_wsum sums
//                them in block order (deterministic) into the gradient.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "qxd_internal.cuh"
#include "trace.cuh"

namespace qxd {

constexpr int PT_SITES = 32;
constexpr int PT_MAXC = 16;
constexpr int WG_THREADS = 256;
constexpr int WG_BLOCKS = 152;  // blocks per path of the weight-gradient kernel

// transported spinor (T_p h)(x) for the site with checkerboard index cb of parity par
__device__ __forceinline__ void ptc_transport(const Geom& g, const float2* __restrict__ W, const float4* __restrict__ h,
                                              int par, uint32_t cb, int p, cplx<float> out[12]) {
  const float4* hp;
  uint32_t src = cb;
  int spar = par;
  float sign = 1.f;
  int mu = 0;
  bool fwd = true;
  if (p > 0) {
    int x[4];
    cb_coords32(g, cb, par, x);
    fwd = p < 5;
    mu = fwd ? p - 1 : p - 5;
    bool cr;
    src = nbr_cb32(g, x, mu, fwd ? +1 : -1, cr);
    spar = 1 - par;
    if (mu == 0 && cr && g.anti) sign = -1.f;
  }
  hp = h + (i64)spar * 6 * g.sv;
  cplx<float> s[12];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float4 q = __ldg(hp + j * g.sv + src);
    s[2 * j] = mk(sign * q.x, sign * q.y);
    s[2 * j + 1] = mk(sign * q.z, sign * q.w);
  }
  if (p == 0) {
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = s[k];
    return;
  }
  // link W_mu(x) (forward, parity par, site cb) or W_mu(x-mu)^+ (backward, parity 1-par, site src)
  const int lp = fwd ? par : 1 - par;
  const uint32_t ls = fwd ? cb : src;
  cplx<float> u[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float2 w = __ldg(W + ((i64)(lp * 4 + mu) * 9 + k) * g.sv + ls);
    u[k] = mk(w.x, w.y);
  }
  if (fwd) {  // separate loops: each path executes only its own products
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        cplx<float> r = mk(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; ++b) r = cmac(r, u[3 * a + b], s[3 * sp + b]);
        out[3 * sp + a] = r;
      }
  } else {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        cplx<float> r = mk(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 3; ++b) r = cjmac(r, u[3 * b + a], s[3 * sp + b]);
        out[3 * sp + a] = r;
      }
  }
}

// out[co] (par, cb) = sum_{ci, p} Om[co][ci][p] (T_p in_ci)(x)
__global__ void __launch_bounds__(PT_SITES* PT_MAXC) k_ptc_layer(Geom g, int cin, int cout, const float4* __restrict__ in,
                                                                const float2* __restrict__ Om, const float2* __restrict__ W,
                                                                float4* __restrict__ out) {
  __shared__ float2 T[PT_MAXC][12][PT_SITES];
  const int s = threadIdx.x, j = threadIdx.y;
  const int par = blockIdx.y;
  const uint32_t cb = blockIdx.x * PT_SITES + s;
  const bool live = cb < (uint32_t)g.Vh;
  const i64 cs = 12 * g.sv;  // channel stride (float4)
  cplx<float> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = mk(0.f, 0.f);
  for (int p = 0; p < 9; ++p) {
    for (int ci = j; ci < cin; ci += cout) {
      cplx<float> t[12];
      if (live) {
        ptc_transport(g, W, in + ci * cs, par, cb, p, t);
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) t[k] = mk(0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) T[ci][k][s] = make_float2(t[k].re, t[k].im);
    }
    __syncthreads();
    for (int ci = 0; ci < cin; ++ci) {
      const float2* om = Om + (((i64)j * cin + ci) * 9 + p) * 16;
      cplx<float> m[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        float2 w = __ldg(om + k);
        m[k] = mk(w.x, w.y);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        cplx<float> tv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          float2 q = T[ci][3 * t + a][s];
          tv[t] = mk(q.x, q.y);
        }
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
          cplx<float> r = acc[3 * sp + a];
#pragma unroll
          for (int t = 0; t < 4; ++t) r = cmac(r, m[4 * sp + t], tv[t]);
          acc[3 * sp + a] = r;
        }
      }
    }
    __syncthreads();
  }
  if (!live) return;
  float4* o = out + j * cs + (i64)par * 6 * g.sv;
#pragma unroll
  for (int q = 0; q < 6; ++q)
    o[q * g.sv + cb] = make_float4(acc[2 * q].re, acc[2 * q].im, acc[2 * q + 1].re, acc[2 * q + 1].im);
}

// Om_adj[ci][co][swap p] = Om[co][ci][p]^+
__global__ void k_ptc_adjoint_weights(int cin, int cout, const float2* __restrict__ Om, float2* __restrict__ Oa) {
  const int n = cout * cin * 9;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int p = e % 9, ci = (e / 9) % cin, co = e / (9 * cin);
    const int ps = p == 0 ? 0 : (p < 5 ? p + 4 : p - 4);
    const float2* src = Om + (i64)e * 16;
    float2* dst = Oa + (((i64)ci * cout + co) * 9 + ps) * 16;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float2 w = src[4 * s + t];
        dst[4 * t + s] = make_float2(w.x, -w.y);
      }
  }
}

// per-block partial dL/dOmega* of one path p = blockIdx.y: entries (co, ci, s, t)
__global__ void __launch_bounds__(WG_THREADS) k_ptc_wgrad(Geom g, int cin, int cout, const float4* __restrict__ h,
                                                        const float4* __restrict__ gr, const float2* __restrict__ W,
                                                        float2* __restrict__ part) {
  __shared__ float2 T[PT_MAXC][12][PT_SITES];
  __shared__ float2 G[PT_MAXC][12][PT_SITES];
  const int p = blockIdx.y;
  const int tid = threadIdx.x;
  const int nent = cout * cin * 16;
  const i64 cs = 12 * g.sv;
  constexpr int MAXE = PT_MAXC * PT_MAXC * 16 / WG_THREADS;  // entries per thread (16 at C = 16)
  cplx<float> acc[MAXE];
#pragma unroll
  for (int k = 0; k < MAXE; ++k) acc[k] = mk(0.f, 0.f);
  const i64 ntiles = 2 * ((g.Vh + PT_SITES - 1) / PT_SITES);  // tiles over both parities
  for (i64 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int par = (int)(tile & 1);
    const uint32_t cb0 = (uint32_t)(tile >> 1) * PT_SITES;
    // stage T_p h_ci and g_co for the tile's 32 sites
    for (int e = tid; e < (cin + cout) * PT_SITES; e += WG_THREADS) {
      const int s = e % PT_SITES, c = e / PT_SITES;
      const uint32_t cb = cb0 + s;
      cplx<float> t[12];
      if (cb < (uint32_t)g.Vh) {
        if (c < cin) {
          ptc_transport(g, W, h + c * cs, par, cb, p, t);
        } else {
          const float4* gp = gr + (c - cin) * cs + (i64)par * 6 * g.sv;
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            float4 v = __ldg(gp + q * g.sv + cb);
            t[2 * q] = mk(v.x, v.y);
            t[2 * q + 1] = mk(v.z, v.w);
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) t[k] = mk(0.f, 0.f);
      }
      if (c < cin) {
#pragma unroll
        for (int k = 0; k < 12; ++k) T[c][k][s] = make_float2(t[k].re, t[k].im);
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) G[c - cin][k][s] = make_float2(t[k].re, t[k].im);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < MAXE; ++k) {
      const int e = tid + k * WG_THREADS;
      if (e < nent) {
        const int t = e % 4, sp = (e / 4) % 4, ci = (e / 16) % cin, co = e / (16 * cin);
        cplx<float> r = acc[k];
        for (int s = 0; s < PT_SITES; ++s)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            float2 gv = G[co][3 * sp + a][s], tv = T[ci][3 * t + a][s];
            r = cjmac(r, mk(tv.x, tv.y), mk(gv.x, gv.y));  // g * conj(T)
          }
        acc[k] = r;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < MAXE; ++k) {
    const int e = tid + k * WG_THREADS;
    if (e < nent) {
      const int t = e % 4, sp = (e / 4) % 4, ci = (e / 16) % cin, co = e / (16 * cin);
      const i64 w = (((i64)co * cin + ci) * 9 + p) * 16 + 4 * sp + t;
      part[(i64)blockIdx.x * cout * cin * 9 * 16 + w] = make_float2(acc[k].re, acc[k].im);
    }
  }
}

// grad[w] += sum over blocks of part[b][w] (block order)
__global__ void k_ptc_wsum(int nw, int nb, const float2* __restrict__ part, double2* __restrict__ grad) {
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int b = 0; b < nb; ++b) {
      float2 v = part[(i64)b * nw + w];
      re += v.x;
      im += v.y;
    }
    grad[w].x += re;
    grad[w].y += im;
  }
}

// Adam on the real and imaginary parts; the real-parameter gradient is 2 Re / 2 Im of dL/dOmega*
__global__ void k_adam(int nw, float2* __restrict__ w, const double2* __restrict__ grad, float2* __restrict__ m,
                       float2* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2, float scale) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
    const float gr = 2.f * (float)grad[i].x * scale, gi = 2.f * (float)grad[i].y * scale;
    float2 mm = m[i], vv = v[i], ww = w[i];
    mm.x = b1 * mm.x + (1.f - b1) * gr;
    mm.y = b1 * mm.y + (1.f - b1) * gi;
    vv.x = b2 * vv.x + (1.f - b2) * gr * gr;
    vv.y = b2 * vv.y + (1.f - b2) * gi * gi;
    ww.x -= lr * (mm.x / c1) / (sqrtf(vv.x / c2) + eps);
    ww.y -= lr * (mm.y / c1) / (sqrtf(vv.y / c2) + eps);
    m[i] = mm;
    v[i] = vv;
    w[i] = ww;
  }
}

// g = y - v over n4 float4 (FP32); returns ||g||^2 through the FP32 norm kernel
__global__ void k_sub32(const float4* __restrict__ y, const float4* __restrict__ v, float4* __restrict__ g, i64 n4) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n4; i += (i64)gridDim.x * blockDim.x) {
    float4 a = y[i], b = v[i];
    g[i] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
  }
}

}  // namespace qxd

using namespace qxd;

struct qxd_net {
  qxd_lattice* lat = nullptr;
  int nlayers = 0;
  int ch[9] = {0};
  i64 woff[9] = {0};  // complex offset of each layer's weights
  i64 nw = 0;         // complex weights in total
  float2* w = nullptr;
  float2* wadj = nullptr;  // adjoint weights of one layer (scratch)
  double2* grad = nullptr;
  float2* am = nullptr;
  float2* av = nullptr;
  float2* part = nullptr;  // wgrad partials
  int adam_t = 0;
  float4* act[9] = {nullptr};   // activations of one sample (layer inputs/outputs)
  float4* gbuf[2] = {nullptr};  // gradient ping-pong buffers (max channels)
  int maxc = 1;
  // inference precision: QXD_NET_BF16_TC (tensor-core channel mix) or QXD_NET_F32
  int prec = QXD_NET_BF16_TC;
  unsigned char* bp = nullptr;  // packed BF16 weights of every layer (tensor-core layout)
  i64 bpoff[9] = {0};           // byte offset of each layer's packed weights
  bool bp_valid = false;        // packed weights match w
  int* tc_err = nullptr;        // error word of the tensor-core kernel
  float4* tc_scratch = nullptr; // virtual channels of pull-form layers
  // the adjoint network M^+ (layers in reverse, each the adjoint layer): its FP32 weights and
  // their tensor-core packing, rebuilt from w when adj_valid is false
  float2* wadj_all = nullptr;
  unsigned char* bpadj = nullptr;
  i64 bpadjoff[9] = {0};
  bool adj_valid = false;
};

namespace qxd {

static int ew_grid(i64 n) {
  i64 b = (n + 255) / 256;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

static qxd_status layer_fwd(qxd_net* net, int l, const float4* in, float4* out, bool adjoint) {
  qxd_lattice* lat = net->lat;
  const int ci = adjoint ? net->ch[l + 1] : net->ch[l];
  const int co = adjoint ? net->ch[l] : net->ch[l + 1];
  const float2* Om = net->w + net->woff[l];
  if (adjoint) {
    k_ptc_adjoint_weights<<<ew_grid(ci * co * 9), 256, 0, lat->stream>>>(net->ch[l], net->ch[l + 1], Om, net->wadj);
    QXD_CHECK_LAUNCH(lat, "k_ptc_adjoint_weights");
    Om = net->wadj;
  }
  dim3 grid((unsigned)((lat->Vh + PT_SITES - 1) / PT_SITES), 2), block(PT_SITES, co);
  prof_begin(lat, KSTAT_PTC_F32, (96.0 * (ci + co) + 576.0) * (double)lat->V);
  k_ptc_layer<<<grid, block, 0, lat->stream>>>(lat->g, ci, co, in, Om, lat->W32, out);
  prof_end(lat);
  QXD_CHECK_LAUNCH(lat, "k_ptc_layer");
  return QXD_OK;
}

// M(in) for one-channel full FP32 fields; uses net->act as scratch.  With QXD_NET_BF16_TC the
// layers run on the tensor cores (weights packed once per weight update).
qxd_status net_apply32(qxd_net* net, const float4* in, float4* out) {
  qxd_status st;
  if (net->prec == QXD_NET_BF16_TC && !net->bp_valid) {
    for (int l = 0; l < net->nlayers; ++l)
      if ((st = ptc_pack_weights(net->lat, net->ch[l], net->ch[l + 1], net->w + net->woff[l], net->bp + net->bpoff[l])))
        return st;
    net->bp_valid = true;
  }
  const float4* h = in;
  for (int l = 0; l < net->nlayers; ++l) {
    float4* o = (l == net->nlayers - 1) ? out : net->act[l + 1];
    if (net->prec == QXD_NET_BF16_TC)  // activations between layers in BF16
      st = ptc_layer_tc(net->lat, net->ch[l], net->ch[l + 1], h, l > 0, net->bp + net->bpoff[l], o,
                        l < net->nlayers - 1, net->tc_scratch, net->tc_err);
    else
      st = layer_fwd(net, l, h, o, false);
    if (st) return st;
    h = o;
  }
  return QXD_OK;
}

// M^+(in): the adjoint network, for the normal-equation solver that uses M as a right
// preconditioner.  The adjoint of a layer with weights Omega[c][c'][p] is the layer from the c
// channels to the c' channels with weights Omega[c][c'][swap p]^+ (the transport of path p has
// the transport of the opposite path as adjoint, and it commutes with the spin matrices); the
// adjoint network runs those layers last to first.  Same precision as net_apply32.
qxd_status net_apply_adj32(qxd_net* net, const float4* in, float4* out) {
  qxd_lattice* lat = net->lat;
  qxd_status st;
  if (!net->adj_valid) {
    for (int l = 0; l < net->nlayers; ++l) {
      const int ci = net->ch[l], co = net->ch[l + 1];
      k_ptc_adjoint_weights<<<ew_grid(ci * co * 9), 256, 0, lat->stream>>>(ci, co, net->w + net->woff[l],
                                                                           net->wadj_all + net->woff[l]);
      QXD_CHECK_LAUNCH(lat, "k_ptc_adjoint_weights");
      if ((st = ptc_pack_weights(lat, co, ci, net->wadj_all + net->woff[l], net->bpadj + net->bpadjoff[l]))) return st;
    }
    net->adj_valid = true;
  }
  const float4* h = in;
  for (int i = 0; i < net->nlayers; ++i) {
    const int l = net->nlayers - 1 - i;
    const int ci = net->ch[l + 1], co = net->ch[l];
    float4* o = (l == 0) ? out : net->act[l];
    if (net->prec == QXD_NET_BF16_TC) {
      st = ptc_layer_tc(lat, ci, co, h, i > 0, net->bpadj + net->bpadjoff[l], o, l > 0, net->tc_scratch, net->tc_err);
    } else {
      dim3 grid((unsigned)((lat->Vh + PT_SITES - 1) / PT_SITES), 2), block(PT_SITES, co);
      prof_begin(lat, KSTAT_PTC_F32, (96.0 * (ci + co) + 576.0) * (double)lat->V);
      k_ptc_layer<<<grid, block, 0, lat->stream>>>(lat->g, ci, co, h, net->wadj_all + net->woff[l], lat->W32, o);
      prof_end(lat);
      QXD_CHECK_LAUNCH(lat, "k_ptc_layer");
      st = QXD_OK;
    }
    if (st) return st;
    h = o;
  }
  return QXD_OK;
}

// error word of the tensor-core kernel (synchronises the lattice stream)
qxd_status net_check(qxd_net* net) {
  if (!net || net->prec != QXD_NET_BF16_TC) return QXD_OK;
  int e = 0;
  QXD_CUDA(net->lat, cudaMemcpyAsync(&e, net->tc_err, sizeof(int), cudaMemcpyDeviceToHost, net->lat->stream));
  QXD_CUDA(net->lat, cudaStreamSynchronize(net->lat->stream));
  if (e) return fail(net->lat, QXD_ETIMEOUT, "a bounded wait of the tensor-core PTC layer expired");
  return QXD_OK;
}

// accumulate dL/dOmega* of one sample into net->grad; returns ||M(b) - v||^2 (FP64)
static qxd_status net_sample_grad(qxd_net* net, const float4* b, const float4* v, double* loss) {
  qxd_lattice* lat = net->lat;
  const i64 cs = 12 * lat->sv;
  // forward, keeping every layer's input
  net->act[0] = const_cast<float4*>(b);
  for (int l = 0; l < net->nlayers; ++l) {
    qxd_status st = layer_fwd(net, l, net->act[l], net->act[l + 1], false);
    if (st) return st;
  }
  // g = y - v, loss
  float4* g = net->gbuf[0];
  k_sub32<<<ew_grid(cs), 256, 0, lat->stream>>>(net->act[net->nlayers], v, g, cs);
  QXD_CHECK_LAUNCH(lat, "k_sub32");
  qxd_status st = blas_norm2_32(lat, g, cs, SC_TMP3);
  if (st) return st;
  st = read_scalars(lat, SC_TMP3, 1, loss);
  if (st) return st;
  int cur = 0;
  for (int l = net->nlayers - 1; l >= 0; --l) {
    const int ci = net->ch[l], co = net->ch[l + 1];
    dim3 grid(WG_BLOCKS, 9);
    k_ptc_wgrad<<<grid, WG_THREADS, 0, lat->stream>>>(lat->g, ci, co, net->act[l], net->gbuf[cur], lat->W32, net->part);
    QXD_CHECK_LAUNCH(lat, "k_ptc_wgrad");
    const int nwl = co * ci * 9 * 16;
    k_ptc_wsum<<<ew_grid(nwl), 256, 0, lat->stream>>>(nwl, WG_BLOCKS, net->part, net->grad + net->woff[l]);
    QXD_CHECK_LAUNCH(lat, "k_ptc_wsum");
    if (l > 0) {
      st = layer_fwd(net, l, net->gbuf[cur], net->gbuf[1 - cur], true);
      if (st) return st;
      cur = 1 - cur;
    }
  }
  return QXD_OK;
}

}  // namespace qxd

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

extern "C" {

qxd_status qxd_net_create(qxd_lattice* lat, int nlayers, const int* channels, uint64_t seed, qxd_net** out) {
  QXD_TRACE();
  if (!lat || !channels || !out) return QXD_EINVAL;
  *out = nullptr;
  if (nlayers < 1 || nlayers > 8) return fail(lat, QXD_EINVAL, "nlayers must be 1..8");
  if (channels[0] != 1 || channels[nlayers] != 1) return fail(lat, QXD_EINVAL, "first and last channel counts must be 1");
  for (int l = 0; l <= nlayers; ++l)
    if (channels[l] < 1 || channels[l] > PT_MAXC) return fail(lat, QXD_EINVAL, "channel counts must be 1..16");
  if (!lat->have_gauge) return fail(lat, QXD_ESTATE, "net_create before load_gauge");
  qxd_net* net = new qxd_net();
  net->lat = lat;
  net->nlayers = nlayers;
  i64 off = 0;
  for (int l = 0; l <= nlayers; ++l) {
    net->ch[l] = channels[l];
    net->maxc = std::max(net->maxc, channels[l]);
  }
  for (int l = 0; l < nlayers; ++l) {
    net->woff[l] = off;
    off += (i64)channels[l] * channels[l + 1] * 9 * 16;
  }
  net->nw = off;
  const i64 cs = 12 * lat->sv;
  bool ok = cudaMalloc(&net->w, sizeof(float2) * off) == cudaSuccess &&
            cudaMalloc(&net->wadj, sizeof(float2) * PT_MAXC * PT_MAXC * 9 * 16) == cudaSuccess &&
            cudaMalloc(&net->grad, sizeof(double2) * off) == cudaSuccess &&
            cudaMalloc(&net->am, sizeof(float2) * off) == cudaSuccess &&
            cudaMalloc(&net->av, sizeof(float2) * off) == cudaSuccess &&
            cudaMalloc(&net->part, sizeof(float2) * PT_MAXC * PT_MAXC * 9 * 16 * WG_BLOCKS) == cudaSuccess &&
            cudaMalloc(&net->tc_err, sizeof(int)) == cudaSuccess;
  i64 bpb = 0;
  for (int l = 0; l < nlayers; ++l) {
    net->bpoff[l] = bpb;
    bpb += (i64)ptc_tc_packed_bytes(channels[l], channels[l + 1]);
  }
  ok = ok && cudaMalloc(&net->bp, (size_t)bpb) == cudaSuccess;
  i64 bpa = 0;  // the adjoint layers (c -> c') packed
  for (int l = 0; l < nlayers; ++l) {
    net->bpadjoff[l] = bpa;
    bpa += (i64)ptc_tc_packed_bytes(channels[l + 1], channels[l]);
  }
  ok = ok && cudaMalloc(&net->bpadj, (size_t)bpa) == cudaSuccess &&
       cudaMalloc(&net->wadj_all, sizeof(float2) * off) == cudaSuccess;
  size_t scr = 0;
  for (int l = 0; l < nlayers; ++l)
    scr = std::max(scr, std::max(ptc_tc_pull_scratch(channels[l], channels[l + 1], lat->sv),
                                 ptc_tc_pull_scratch(channels[l + 1], channels[l], lat->sv)));
  if (scr) ok = ok && cudaMalloc(&net->tc_scratch, sizeof(float4) * scr) == cudaSuccess;
  if (ok) cudaMemsetAsync(net->tc_err, 0, sizeof(int), lat->stream);
  for (int l = 1; l <= nlayers && ok; ++l) ok = cudaMalloc(&net->act[l], sizeof(float4) * cs * channels[l]) == cudaSuccess;
  for (int k = 0; k < 2 && ok; ++k) ok = cudaMalloc(&net->gbuf[k], sizeof(float4) * cs * net->maxc) == cudaSuccess;
  if (!ok) {
    qxd_net_destroy(net);
    return fail(lat, QXD_ENOMEM, "net allocation failed");
  }
  cudaMemsetAsync(net->am, 0, sizeof(float2) * off, lat->stream);
  cudaMemsetAsync(net->av, 0, sizeof(float2) * off, lat->stream);
  for (int k = 0; k < 2; ++k) cudaMemsetAsync(net->gbuf[k], 0, sizeof(float4) * cs * net->maxc, lat->stream);
  // initial weights: identity path near the point-Jacobi scale 1/(4+m0) (through the channel
  // chain), small seeded noise elsewhere
  std::vector<float2> h(off);
  for (int l = 0; l < nlayers; ++l) {
    const int ci = channels[l], co = channels[l + 1];
    const double diag = l == 0 ? 0.25 / ci : 1.0 / ci;  // product over layers ~ 0.25 on the identity
    for (i64 e = 0; e < (i64)ci * co * 9 * 16; ++e) {
      const int t = (int)(e % 4), s = (int)((e / 4) % 4), p = (int)((e / 16) % 9);
      uint64_t z1 = mix64(seed + (uint64_t)(net->woff[l] + e) * 2 * 0x9E3779B97F4A7C15ull + 0x9E3779B97F4A7C15ull);
      uint64_t z2 = mix64(seed + (uint64_t)(net->woff[l] + e) * 2 * 0x9E3779B97F4A7C15ull + 2 * 0x9E3779B97F4A7C15ull);
      double u1 = (double)(z1 >> 11) * 0x1.0p-53 - 0.5, u2 = (double)(z2 >> 11) * 0x1.0p-53 - 0.5;
      double re = 0.02 * u1, im = 0.02 * u2;
      if (p == 0 && s == t) re += diag;
      h[net->woff[l] + e] = make_float2((float)re, (float)im);
    }
  }
  cudaMemcpyAsync(net->w, h.data(), sizeof(float2) * off, cudaMemcpyHostToDevice, lat->stream);
  if (cudaStreamSynchronize(lat->stream) != cudaSuccess) {
    qxd_net_destroy(net);
    return fail(lat, QXD_ECUDA, "net initialisation failed");
  }
  *out = net;
  return QXD_OK;
}

qxd_status qxd_net_destroy(qxd_net* net) {
  QXD_TRACE();
  if (!net) return QXD_OK;
  if (net->lat) cudaStreamSynchronize(net->lat->stream);
  void* b[] = {net->w,     net->wadj,       net->grad,   net->am,     net->av,     net->part,    net->gbuf[0],
               net->gbuf[1], net->bp,        net->tc_err, net->tc_scratch, net->bpadj, net->wadj_all};
  for (void* p : b)
    if (p) cudaFree(p);
  for (int l = 1; l <= net->nlayers; ++l)
    if (net->act[l]) cudaFree(net->act[l]);
  delete net;
  return QXD_OK;
}

int64_t qxd_net_num_weights(const qxd_net* net) { return net ? net->nw : 0; }

// FP64 boundary field -> FP32 internal full field (uses the API staging slots)
static qxd_status to_internal32(qxd_lattice* lat, const double* src, int on_device, float4* dst) {
  const size_t vb = sizeof(double) * 24 * lat->V;
  double2* f64;
  qxd_status st = ensure_work(lat, 24, sizeof(double2) * 24 * lat->sv, (void**)&f64);
  if (st) return st;
  if (!on_device) {
    void* bi;
    if ((st = ensure_work(lat, 26, vb, &bi))) return st;
    QXD_CUDA(lat, cudaMemcpyAsync(bi, src, vb, cudaMemcpyHostToDevice, lat->stream));
    src = (const double*)bi;
  }
  if ((st = pack_spinor64(lat, (const double2*)src, f64, 0))) return st;
  return f64_to_f32(lat, f64, dst, 12 * lat->sv);
}

static qxd_status from_internal32(qxd_lattice* lat, const float4* src, int on_device, double* dst) {
  const size_t vb = sizeof(double) * 24 * lat->V;
  double2* f64;
  qxd_status st = ensure_work(lat, 25, sizeof(double2) * 24 * lat->sv, (void**)&f64);
  if (st) return st;
  if ((st = f32_to_f64(lat, src, f64, 12 * lat->sv))) return st;
  if (on_device) return unpack_spinor64(lat, f64, (double2*)dst, 0);
  void* bo;
  if ((st = ensure_work(lat, 27, vb, &bo))) return st;
  if ((st = unpack_spinor64(lat, f64, (double2*)bo, 0))) return st;
  QXD_CUDA(lat, cudaMemcpyAsync(dst, bo, vb, cudaMemcpyDeviceToHost, lat->stream));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  return QXD_OK;
}

qxd_status qxd_net_apply_adjoint(qxd_net* net, double* out, const double* in, int on_device) {
  QXD_TRACE();
  if (!net || !out || !in) return QXD_EINVAL;
  qxd_lattice* lat = net->lat;
  float4 *a, *b;
  const size_t fb = sizeof(float4) * 12 * lat->sv;
  qxd_status st;
  if ((st = ensure_work(lat, 39, 2 * fb, (void**)&a))) return st;
  b = a + 12 * lat->sv;
  if ((st = to_internal32(lat, in, on_device, a))) return st;
  if ((st = net_apply_adj32(net, a, b))) return st;
  if ((st = net_check(net))) return st;
  return from_internal32(lat, b, on_device, out);
}

qxd_status qxd_net_apply(qxd_net* net, double* out, const double* in, int on_device) {
  QXD_TRACE();
  if (!net || !out || !in) return QXD_EINVAL;
  qxd_lattice* lat = net->lat;
  float4 *a, *b;
  const size_t fb = sizeof(float4) * 12 * lat->sv;
  qxd_status st;
  if ((st = ensure_work(lat, 39, 2 * fb, (void**)&a))) return st;
  b = a + 12 * lat->sv;
  if ((st = to_internal32(lat, in, on_device, a))) return st;
  if ((st = net_apply32(net, a, b))) return st;
  if ((st = net_check(net))) return st;
  return from_internal32(lat, b, on_device, out);
}

qxd_status qxd_net_loss_grad(qxd_net* net, const double* v, const double* b, int nsamp, int on_device, double* loss,
                             double* grad) {
  QXD_TRACE();
  if (!net || !v || !b || nsamp <= 0 || !loss) return QXD_EINVAL;
  qxd_lattice* lat = net->lat;
  const i64 cs = 12 * lat->sv;
  float4 *vb32;
  qxd_status st;
  if ((st = ensure_work(lat, 39, 2 * sizeof(float4) * cs, (void**)&vb32))) return st;
  float4* bb32 = vb32 + cs;
  QXD_CUDA(lat, cudaMemsetAsync(net->grad, 0, sizeof(double2) * net->nw, lat->stream));
  double total = 0.0;
  for (int i = 0; i < nsamp; ++i) {
    if ((st = to_internal32(lat, v + (i64)i * 24 * lat->V, on_device, vb32))) return st;
    if ((st = to_internal32(lat, b + (i64)i * 24 * lat->V, on_device, bb32))) return st;
    double l;
    if ((st = net_sample_grad(net, bb32, vb32, &l))) return st;
    total += l;
  }
  *loss = total;
  if (grad) {
    QXD_CUDA(lat, cudaMemcpyAsync(grad, net->grad, sizeof(double2) * net->nw, cudaMemcpyDeviceToHost, lat->stream));
    QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  }
  return QXD_OK;
}

// Adam epochs over a resident training set set[2i] = v_i, set[2i+1] = b_i (FP32, internal layout)
static qxd_status train_on_set(qxd_net* net, const float4* set, int nsamp, const qxd_train_params* p,
                               double* loss_hist) {
  qxd_lattice* lat = net->lat;
  const i64 cs = 12 * lat->sv;
  qxd_status st;
  const float b1 = (float)p->beta1, b2 = (float)p->beta2, eps = (float)p->eps;
  for (int e = 0; e < p->epochs; ++e) {
    double epoch_loss = 0.0;
    for (int s0 = 0; s0 < nsamp; s0 += p->batch) {
      const int s1 = std::min(nsamp, s0 + p->batch);
      QXD_CUDA(lat, cudaMemsetAsync(net->grad, 0, sizeof(double2) * net->nw, lat->stream));
      for (int i = s0; i < s1; ++i) {
        double l;
        if ((st = net_sample_grad(net, set + (i64)(2 * i + 1) * cs, set + (i64)(2 * i) * cs, &l))) return st;
        epoch_loss += l;
      }
      net->adam_t += 1;
      const float c1 = 1.f - powf(b1, (float)net->adam_t), c2 = 1.f - powf(b2, (float)net->adam_t);
      k_adam<<<ew_grid(net->nw), 256, 0, lat->stream>>>((int)net->nw, net->w, net->grad, net->am, net->av,
                                                        (float)p->lr, b1, b2, eps, c1, c2, 1.f / (float)(s1 - s0));
      QXD_CHECK_LAUNCH(lat, "k_adam");
      net->bp_valid = false;
      net->adj_valid = false;
    }
    if (loss_hist) loss_hist[e] = epoch_loss / nsamp;
  }
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  return QXD_OK;
}

// b_i = D v_i with the FP32 operator, for every sample of a resident training set
static qxd_status make_targets(qxd_lattice* lat, float4* set, int nsamp) {
  const i64 cs = 12 * lat->sv;
  qxd_status st;
  for (int i = 0; i < nsamp; ++i) {
    float4 *vi = set + (i64)(2 * i) * cs, *bi = vi + cs;
    if ((st = hop32(lat, 0, EPI_DFULL, 0, vi + 6 * lat->sv, vi, bi, 0.f))) return st;
    if ((st = hop32(lat, 1, EPI_DFULL, 0, vi, vi + 6 * lat->sv, bi + 6 * lat->sv, 0.f))) return st;
  }
  return QXD_OK;
}

static qxd_status check_train(qxd_lattice* lat, const qxd_train_params* p) {
  if (p->version != 1 && p->version != QXD_TRAIN_VERSION) return fail(lat, QXD_EINVAL, "qxd_train_params version mismatch");
  if (p->epochs <= 0 || p->batch <= 0 || !(p->lr > 0)) return fail(lat, QXD_EINVAL, "epochs, batch, lr must be > 0");
  if (!lat->have_clover) return fail(lat, QXD_ESTATE, "train before build_clover");
  return QXD_OK;
}

qxd_status qxd_net_train(qxd_net* net, const double* v, int nsamp, const qxd_train_params* p, double* loss_hist,
                         int on_device) {
  QXD_TRACE();
  if (!net || !v || !p || nsamp <= 0) return QXD_EINVAL;
  qxd_lattice* lat = net->lat;
  qxd_status st;
  if ((st = check_train(lat, p))) return st;
  const i64 cs = 12 * lat->sv;
  // training set: v_i and b_i = D v_i (FP32 operator), kept resident in FP32
  float4* set;
  if ((st = ensure_work(lat, 31, sizeof(float4) * cs * 2 * nsamp, (void**)&set))) return st;
  // the slot is shared with other solvers: clear the padding lanes the kernels below never write
  QXD_CUDA(lat, cudaMemsetAsync(set, 0, sizeof(float4) * cs * 2 * nsamp, lat->stream));
  for (int i = 0; i < nsamp; ++i)
    if ((st = to_internal32(lat, v + (i64)i * 24 * lat->V, on_device, set + (i64)(2 * i) * cs))) return st;
  if ((st = make_targets(lat, set, nsamp))) return st;
  return train_on_set(net, set, nsamp, p, loss_hist);
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used counter-style: output i of the stream with
// seed s is mix64(s + (i + 1) * golden ratio constant); uniforms are the top 53 bits.
__device__ __forceinline__ double sm64_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

// Gaussian training sample: component k = 3 alpha + a of the site with lexicographic index x
// (Eq. lexi, on the device lattice) is (r cos th, r sin th) by Box-Muller from uniforms 2j and
// 2j + 1 of the stream, j = 12 x + k, r = sqrt(-2 log(1 - u1)), th = 2 pi u2; written in the
// internal FP32 layout (both parities).
__global__ void k_gauss_spinor32(Geom g, uint64_t seed, float4* __restrict__ out) {
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * g.Vh) return;
  const int par = t >= g.Vh ? 1 : 0;
  const uint32_t cb = (uint32_t)(t - par * g.Vh);
  int x[4];
  cb_coords32(g, cb, par, x);
  const uint64_t lex = (((uint64_t)x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
  float4* o = out + (i64)par * 6 * g.sv + cb;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    float c[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint64_t pair = 12 * lex + 2 * j + h;
      const double u1 = sm64_uniform(seed, 2 * pair), u2 = sm64_uniform(seed, 2 * pair + 1);
      const double r = sqrt(-2.0 * log1p(-u1));
      double sn, cs;
      sincos(6.283185307179586 * u2, &sn, &cs);
      c[2 * h] = (float)(r * cs);
      c[2 * h + 1] = (float)(r * sn);
    }
    o[(i64)j * g.sv] = make_float4(c[0], c[1], c[2], c[3]);
  }
}

qxd_status qxd_train_precond(qxd_lattice* lat, const qxd_train_params* p, qxd_net** out) {
  QXD_TRACE();
  if (!lat || !p || !out) return QXD_EINVAL;
  *out = nullptr;
  if (p->version != QXD_TRAIN_VERSION) return fail(lat, QXD_EINVAL, "qxd_train_precond needs qxd_train_params version 2");
  qxd_status st;
  if ((st = check_train(lat, p))) return st;
  if (p->nsamp <= 0) return fail(lat, QXD_EINVAL, "nsamp must be > 0");
  qxd_net* net = nullptr;
  if ((st = qxd_net_create(lat, p->nlayers, p->channels, p->net_seed, &net))) return st;
  const i64 cs = 12 * lat->sv;
  float4* set;
  st = ensure_work(lat, 31, sizeof(float4) * cs * 2 * p->nsamp, (void**)&set);
  if (st == QXD_OK) {  // padding lanes stay zero, as after to_internal32
    const cudaError_t e = cudaMemsetAsync(set, 0, sizeof(float4) * cs * 2 * p->nsamp, lat->stream);
    if (e != cudaSuccess) st = cuda_fail(lat, e, "cudaMemsetAsync");
  }
  for (int i = 0; i < p->nsamp && st == QXD_OK; ++i) {
    const unsigned grid = (unsigned)((2 * lat->g.Vh + 255) / 256);
    k_gauss_spinor32<<<grid, 256, 0, lat->stream>>>(lat->g, p->sample_seed + (uint64_t)i, set + (i64)(2 * i) * cs);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
      st = cuda_fail(lat, e, "k_gauss_spinor32");
    else
      lat->launches++;
  }
  if (st == QXD_OK) st = make_targets(lat, set, p->nsamp);
  if (st == QXD_OK) st = train_on_set(net, set, p->nsamp, p, p->loss_hist);
  if (st != QXD_OK) {
    qxd_net_destroy(net);
    return st;
  }
  *out = net;
  return QXD_OK;
}

// file: "QXDNET1\n", then int32 nlayers, int32 channels[nlayers+1], float32 weights (re, im)
qxd_status qxd_net_save(const qxd_net* net, const char* path) {
  QXD_TRACE();
  if (!net || !path) return QXD_EINVAL;
  std::vector<double> w(2 * net->nw);
  qxd_status st = qxd_net_get_weights(net, w.data());
  if (st) return st;
  FILE* f = fopen(path, "wb");
  if (!f) return fail(net->lat, QXD_EINVAL, "cannot open the net file for writing");
  const char magic[8] = {'Q', 'X', 'D', 'N', 'E', 'T', '1', '\n'};
  int32_t nl = net->nlayers, ch[9];
  for (int l = 0; l <= net->nlayers; ++l) ch[l] = net->ch[l];
  bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(&nl, 4, 1, f) == 1 && fwrite(ch, 4, nl + 1, f) == (size_t)(nl + 1);
  for (i64 i = 0; i < 2 * net->nw && ok; ++i) {
    float x = (float)w[i];
    ok = fwrite(&x, 4, 1, f) == 1;
  }
  fclose(f);
  return ok ? QXD_OK : fail(net->lat, QXD_EINVAL, "short write of the net file");
}

qxd_status qxd_net_load(qxd_lattice* lat, const char* path, qxd_net** out) {
  QXD_TRACE();
  if (!lat || !path || !out) return QXD_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(lat, QXD_EINVAL, "cannot open the net file");
  char magic[8];
  int32_t nl = 0, ch[9];
  bool ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "QXDNET1\n", 8) == 0 && fread(&nl, 4, 1, f) == 1 &&
            nl >= 1 && nl <= 8 && fread(ch, 4, nl + 1, f) == (size_t)(nl + 1);
  if (!ok) {
    fclose(f);
    return fail(lat, QXD_EINVAL, "not a qxd net file");
  }
  int chi[9];
  for (int l = 0; l <= nl; ++l) chi[l] = ch[l];
  qxd_status st = qxd_net_create(lat, nl, chi, 0, out);
  if (st) {
    fclose(f);
    return st;
  }
  std::vector<double> w(2 * (*out)->nw);
  for (i64 i = 0; i < 2 * (*out)->nw && ok; ++i) {
    float x;
    ok = fread(&x, 4, 1, f) == 1;
    w[i] = x;
  }
  fclose(f);
  if (!ok) {
    qxd_net_destroy(*out);
    *out = nullptr;
    return fail(lat, QXD_EINVAL, "truncated net file");
  }
  return qxd_net_set_weights(*out, w.data());
}

qxd_status qxd_net_set_weights(qxd_net* net, const double* w) {
  if (!net || !w) return QXD_EINVAL;
  std::vector<float2> h(net->nw);
  for (i64 i = 0; i < net->nw; ++i) h[i] = make_float2((float)w[2 * i], (float)w[2 * i + 1]);
  QXD_CUDA(net->lat, cudaMemcpyAsync(net->w, h.data(), sizeof(float2) * net->nw, cudaMemcpyHostToDevice, net->lat->stream));
  QXD_CUDA(net->lat, cudaStreamSynchronize(net->lat->stream));
  net->bp_valid = false;
  net->adj_valid = false;
  return QXD_OK;
}

qxd_status qxd_net_set_precision(qxd_net* net, int prec) {
  if (!net) return QXD_EINVAL;
  if (prec != QXD_NET_F32 && prec != QXD_NET_BF16_TC) return fail(net->lat, QXD_EINVAL, "unknown net precision");
  net->prec = prec;
  return QXD_OK;
}

qxd_status qxd_net_get_weights(const qxd_net* net, double* w) {
  if (!net || !w) return QXD_EINVAL;
  std::vector<float2> h(net->nw);
  QXD_CUDA(net->lat, cudaMemcpyAsync(h.data(), net->w, sizeof(float2) * net->nw, cudaMemcpyDeviceToHost, net->lat->stream));
  QXD_CUDA(net->lat, cudaStreamSynchronize(net->lat->stream));
  for (i64 i = 0; i < net->nw; ++i) {
    w[2 * i] = h[i].x;
    w[2 * i + 1] = h[i].y;
  }
  return QXD_OK;
}

}  // extern "C"
