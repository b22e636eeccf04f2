// Boundary <-> device layout transforms and gauge-field ingest (Sec. 4.1: field reordering,
// Sec. 4.2: C* mirror, Sec. 4.3: U(3) hop links).
//
// Boundary site orders (pure index functions, no lookup arrays, as Sec. 4.1.1 recommends):
//   LEXI: boundary index = Lambda(x, L).  IPT: Eq. ipt with the lattice's cache blocks B
//   (ipt_index / ipt_coords; B = L gives cb + P(x) V/2).
// Both map onto the device's (parity, cb = floor(Lambda/2)) addressing.
#include "df64.cuh"
#include "qxd_internal.cuh"

namespace qxd {

// (parity, cb) of the site with boundary index i.
__device__ __forceinline__ void bnd_to_pc(const Geom& g, int order, i64 i, int& par, i64& cb) {
  if (order == QXD_ORDER_IPT) {
    int x[4];
    ipt_coords(g.L, g.B, i, x);
    par = (x[0] + x[1] + x[2] + x[3]) & 1;
    cb = lexi(g, x) >> 1;
  } else {
    i64 t = i;
    int x3 = (int)(t % g.L[3]);
    t /= g.L[3];
    int x2 = (int)(t % g.L[2]);
    t /= g.L[2];
    int x1 = (int)(t % g.L[1]);
    int x0 = (int)(t / g.L[1]);
    par = (x0 + x1 + x2 + x3) & 1;
    cb = i >> 1;
  }
}

// Boundary spinor [N][12] double2 -> device field.  half_only: N = Vh sites of parity 0 in
// cb order, written into a single-parity field [12][sv]; else N = V into [2][12][sv].
__global__ void k_pack_spinor(Geom g, int order, int half_only, const double2* __restrict__ bnd,
                              double2* __restrict__ field) {
  i64 n = (half_only ? g.Vh : 2 * g.Vh) * 12;
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    i64 site = t / 12;
    int k = (int)(t - site * 12);
    int par;
    i64 cb;
    if (half_only) {
      par = 0;
      cb = site;
    } else {
      bnd_to_pc(g, order, site, par, cb);
    }
    field[((i64)par * 12 + k) * g.sv + cb] = bnd[t];
  }
}

__global__ void k_unpack_spinor(Geom g, int order, int half_only, const double2* __restrict__ field,
                                double2* __restrict__ bnd) {
  i64 n = (half_only ? g.Vh : 2 * g.Vh) * 12;
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    i64 site = t / 12;
    int k = (int)(t - site * 12);
    int par;
    i64 cb;
    if (half_only) {
      par = 0;
      cb = site;
    } else {
      bnd_to_pc(g, order, site, par, cb);
    }
    bnd[t] = field[((i64)par * 12 + k) * g.sv + cb];
  }
}

static int grid_cap(i64 n, int bs) {
  i64 b = (n + bs - 1) / bs;
  return (int)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}

qxd_status pack_spinor64(qxd_lattice* lat, const double2* bnd, double2* field, int half_only) {
  i64 n = (half_only ? lat->Vh : lat->V) * 12;
  k_pack_spinor<<<grid_cap(n, 256), 256, 0, lat->stream>>>(lat->g, lat->order, half_only, bnd, field);
  QXD_CHECK_LAUNCH(lat, "k_pack_spinor");
  return QXD_OK;
}

qxd_status unpack_spinor64(qxd_lattice* lat, const double2* field, double2* bnd, int half_only) {
  i64 n = (half_only ? lat->Vh : lat->V) * 12;
  k_unpack_spinor<<<grid_cap(n, 256), 256, 0, lat->stream>>>(lat->g, lat->order, half_only, field, bnd);
  QXD_CHECK_LAUNCH(lat, "k_unpack_spinor");
  return QXD_OK;
}

// Gauge ingest.  One thread per (device site, mu).  The source site on the physical lattice is
// the site itself, or for C* mirror sites (x1 >= shift) the site x1 - shift, whose link is
// conjugated and whose angle changes sign (Sec. 4.2).  Hop link W = exp(i q A) U (Sec. 4.3).
__global__ void k_ingest_gauge(Geom g, int order, int Lp1, int Lp2, int Lp3, i64 Vph,
                               const double2* __restrict__ su3, const double* __restrict__ a, double q,
                               float4* __restrict__ U, double* __restrict__ A, double2* __restrict__ W) {
  i64 n = 2 * g.Vh * 4;
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    int mu = (int)(t & 3);
    i64 s = t >> 2;
    int par = s >= g.Vh ? 1 : 0;
    i64 cb = s - (i64)par * g.Vh;
    int x[4];
    cb_coords(g, cb, par, x);
    bool mirror = false;
    if (g.shift && x[1] >= g.shift) {
      mirror = true;
      x[1] -= g.shift;
    }
    i64 lam = (((i64)x[0] * Lp1 + x[1]) * Lp2 + x[2]) * Lp3 + x[3];
    i64 src;
    if (order == QXD_ORDER_IPT) {
      const int Lp[4] = {g.L[0], Lp1, Lp2, Lp3};  // the physical lattice
      int Bp[4];  // one block of the device lattice (the default) is one block of the physical one
#pragma unroll
      for (int m = 0; m < 4; ++m) Bp[m] = g.B[m] == g.L[m] ? Lp[m] : g.B[m];
      src = ipt_index(Lp, Bp, x);
    } else {
      src = lam;
    }
    (void)Vph;
    double ang = a ? a[src * 4 + mu] : 0.0;
    if (mirror) ang = -ang;
    double sn, cs;
    sincos(q * ang, &sn, &cs);
    i64 base = ((i64)(par * 4 + mu) * 9) * g.sv + cb;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 u = su3[(src * 4 + mu) * 9 + k];
      if (mirror) u.y = -u.y;
      U[base + k * g.sv] = cdf_split(u.x, u.y);
      W[base + k * g.sv] = make_double2(cs * u.x - sn * u.y, cs * u.y + sn * u.x);
    }
    A[(i64)(par * 4 + mu) * g.sv + cb] = ang;
  }
}

// Gauge ingest from the openQxD storage: for the odd site x with boundary index x^ (Eq. ipt of
// this lattice), entry 8 (x^ - V/2) + 2 mu holds U_mu(x) and entry 8 (x^ - V/2) + 2 mu + 1 holds
// U_mu(x - mu), x - mu the lattice neighbour with the C* shift (every link has exactly one odd
// end).  The field is the lattice's own (for C* the
// doubled lattice, mirror half included): no mirroring here.  One thread per (device site, mu).
__global__ void k_ingest_openqxd(Geom g, const double2* __restrict__ u8, const double* __restrict__ a8, double q,
                                 float4* __restrict__ U, double* __restrict__ A, double2* __restrict__ W) {
  const i64 n = 2 * g.Vh * 4;
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    const int mu = (int)(t & 3);
    const i64 s = t >> 2;
    const int par = s >= g.Vh ? 1 : 0;
    const i64 cb = s - (i64)par * g.Vh;
    int x[4];
    cb_coords(g, cb, par, x);
    int y[4] = {x[0], x[1], x[2], x[3]};
    int slot = 2 * mu;
    if (par == 0) {  // even site: its forward link is the backward link of its neighbour x + mu
      const bool crossed = y[mu] + 1 == g.L[mu];
      y[mu] = crossed ? 0 : y[mu] + 1;
      if (crossed && g.shift && mu >= 2) y[1] = (y[1] + g.shift) % g.L[1];  // C*: lands on the mirror copy
      slot += 1;
    }
    const i64 e = (ipt_index(g.L, g.B, y) - g.Vh) * 8 + slot;
    const double ang = a8 ? a8[e] : 0.0;
    double sn, cs;
    sincos(q * ang, &sn, &cs);
    const i64 base = ((i64)(par * 4 + mu) * 9) * g.sv + cb;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double2 u = u8[e * 9 + k];
      U[base + k * g.sv] = cdf_split(u.x, u.y);
      W[base + k * g.sv] = make_double2(cs * u.x - sn * u.y, cs * u.y + sn * u.x);
    }
    A[(i64)(par * 4 + mu) * g.sv + cb] = ang;
  }
}

qxd_status ingest_gauge_openqxd(qxd_lattice* lat, const double2* u8, const double* a8) {
  i64 n = 2 * lat->Vh * 4;
  k_ingest_openqxd<<<grid_cap(n, 128), 128, 0, lat->stream>>>(lat->g, u8, a8, lat->q, lat->U, lat->A, lat->W64);
  QXD_CHECK_LAUNCH(lat, "k_ingest_openqxd");
  return QXD_OK;
}

qxd_status ingest_gauge(qxd_lattice* lat, const double2* su3, const double* a) {
  i64 n = 2 * lat->Vh * 4;
  k_ingest_gauge<<<grid_cap(n, 128), 128, 0, lat->stream>>>(lat->g, lat->order, lat->Lphys[1], lat->Lphys[2],
                                                            lat->Lphys[3], lat->Vphys, su3, a, lat->q, lat->U,
                                                            lat->A, lat->W64);
  QXD_CHECK_LAUNCH(lat, "k_ingest_gauge");
  return QXD_OK;
}

// Link update on the device (the resident field changes in place, no host transfer).  Link j is
// entry idx[j] = 4 s + mu of the canonical arrays load_gauge took (s: the physical site in the
// lattice's site order); its new value is su3[j] (3x3 row-major) and a[j] (or 0 without angles).
// Every device copy of the link (two with C*: the site and its mirror, conjugated with the angle
// negated) gets U, A and the hop link W = exp(i q A) U in FP64, FP32 and both 16-bit formats, and
// the clover sites whose plaquettes hold the link are marked in mask[par * Vh + cb]: the link's
// two end points x and x + mu, each also shifted by +-nu for every nu != mu.  An index outside
// the lattice sets *bad and is skipped.
__device__ __forceinline__ void mark_site(const Geom& g, int y[4], unsigned char* mask) {
  const int par = (y[0] + y[1] + y[2] + y[3]) & 1;
  mask[(i64)par * g.Vh + (lexi(g, y) >> 1)] = 1;
}

__device__ __forceinline__ void shift_site(const Geom& g, int y[4], int mu, int dir) {
  y[mu] += dir;
  bool crossed = false;
  if (y[mu] >= g.L[mu]) {
    y[mu] = 0;
    crossed = true;
  } else if (y[mu] < 0) {
    y[mu] = g.L[mu] - 1;
    crossed = true;
  }
  if (crossed && g.shift && mu >= 2) {
    y[1] += g.shift;
    if (y[1] >= g.L[1]) y[1] -= g.L[1];
  }
}

__global__ void k_update_links(Geom g, int order, int Lp1, int Lp2, int Lp3, i64 n, const int64_t* __restrict__ idx,
                               const double2* __restrict__ su3, const double* __restrict__ a, double q,
                               float4* __restrict__ U, double* __restrict__ A, double2* __restrict__ W,
                               float2* __restrict__ W32, uint32_t* __restrict__ W16, uint32_t* __restrict__ WB16,
                               unsigned char* __restrict__ mask, int* __restrict__ bad) {
  const int Lp[4] = {g.L[0], Lp1, Lp2, Lp3};
  const i64 Vp = (i64)Lp[0] * Lp1 * Lp2 * Lp3;
  for (i64 j = blockIdx.x * (i64)blockDim.x + threadIdx.x; j < n; j += (i64)gridDim.x * blockDim.x) {
    const int64_t e = idx[j];
    if (e < 0 || e >= 4 * Vp) {
      atomicOr(bad, 1);
      continue;
    }
    const int mu = (int)(e & 3);
    const i64 src = e >> 2;
    int x[4];
    if (order == QXD_ORDER_IPT) {
      int Bp[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) Bp[m] = g.B[m] == g.L[m] ? Lp[m] : g.B[m];
      ipt_coords(Lp, Bp, src, x);
    } else {
      i64 t = src;
      x[3] = (int)(t % Lp3);
      t /= Lp3;
      x[2] = (int)(t % Lp2);
      t /= Lp2;
      x[1] = (int)(t % Lp1);
      x[0] = (int)(t / Lp1);
    }
    const double ang0 = a ? a[j] : 0.0;
    for (int copy = 0; copy < (g.shift ? 2 : 1); ++copy) {
      int y[4] = {x[0], x[1] + copy * g.shift, x[2], x[3]};  // copy 1: the C* mirror
      const double ang = copy ? -ang0 : ang0;
      double sn, cs;
      sincos(q * ang, &sn, &cs);
      const int par = (y[0] + y[1] + y[2] + y[3]) & 1;
      const i64 cb = lexi(g, y) >> 1;
      const i64 base = ((i64)(par * 4 + mu) * 9) * g.sv + cb;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        double2 u = su3[j * 9 + k];
        if (copy) u.y = -u.y;
        const double2 w = make_double2(cs * u.x - sn * u.y, cs * u.y + sn * u.x);
        U[base + k * g.sv] = cdf_split(u.x, u.y);
        W[base + k * g.sv] = w;
        W32[base + k * g.sv] = make_float2((float)w.x, (float)w.y);
        const i64 l16 = link16_index(par * 4 + mu, g.sv, k, cb);
        W16[l16] = H16::pack((float)w.x, (float)w.y);
        WB16[l16] = B16::pack((float)w.x, (float)w.y);
      }
      A[(i64)(par * 4 + mu) * g.sv + cb] = ang;
      for (int end = 0; end < 2; ++end) {
        int z[4] = {y[0], y[1], y[2], y[3]};
        if (end) shift_site(g, z, mu, +1);
        mark_site(g, z, mask);
        for (int nu = 0; nu < 4; ++nu) {
          if (nu == mu) continue;
          int zp[4] = {z[0], z[1], z[2], z[3]}, zm[4] = {z[0], z[1], z[2], z[3]};
          shift_site(g, zp, nu, +1);
          shift_site(g, zm, nu, -1);
          mark_site(g, zp, mask);
          mark_site(g, zm, mask);
        }
      }
    }
  }
}

// Marked sites -> a list of par * Vh + cb (order immaterial); *count must start at 0.
__global__ void k_compact_mask(i64 n, const unsigned char* __restrict__ mask, uint32_t* __restrict__ list,
                               unsigned int* __restrict__ count) {
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x)
    if (mask[t]) list[atomicAdd(count, 1u)] = (uint32_t)t;
}

qxd_status update_links(qxd_lattice* lat, i64 n, const int64_t* idx, const double2* su3, const double* a,
                        unsigned char* mask, int* bad) {
  k_update_links<<<grid_cap(n, 128), 128, 0, lat->stream>>>(lat->g, lat->order, lat->Lphys[1], lat->Lphys[2],
                                                            lat->Lphys[3], n, idx, su3, a, lat->q, lat->U, lat->A,
                                                            lat->W64, lat->W32, lat->W16, lat->WB16, mask, bad);
  QXD_CHECK_LAUNCH(lat, "k_update_links");
  return QXD_OK;
}

qxd_status compact_mask(qxd_lattice* lat, const unsigned char* mask, uint32_t* list, unsigned int* count) {
  const i64 n = 2 * lat->Vh;
  k_compact_mask<<<grid_cap(n, 256), 256, 0, lat->stream>>>(n, mask, list, count);
  QXD_CHECK_LAUNCH(lat, "k_compact_mask");
  return QXD_OK;
}

// FP64 hop links -> FP32 and the two 16-bit formats (unitary links need no scale; the 16-bit
// links in the grouped layout of link16_index).
__global__ void k_links_low(i64 n, i64 sv, const double2* __restrict__ W, float2* __restrict__ W32,
                            uint32_t* __restrict__ W16, uint32_t* __restrict__ WB16) {
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    double2 w = W[t];
    W32[t] = make_float2((float)w.x, (float)w.y);
    const i64 pm = t / (9 * sv), k = (t / sv) % 9, cb = t % sv;
    const i64 l16 = link16_index(pm, sv, (int)k, cb);
    W16[l16] = H16::pack((float)w.x, (float)w.y);
    WB16[l16] = B16::pack((float)w.x, (float)w.y);
  }
}

qxd_status convert_links_low(qxd_lattice* lat) {
  i64 n = 2 * 4 * 9 * lat->sv;
  k_links_low<<<grid_cap(n, 256), 256, 0, lat->stream>>>(n, lat->sv, lat->W64, lat->W32, lat->W16, lat->WB16);
  QXD_CHECK_LAUNCH(lat, "k_links_low");
  return QXD_OK;
}

// FP64 planes [2m][sv] double2 -> FP32 planes [m][sv] float4 (pairs of components), n = m * sv.
__global__ void k_f64_to_f32(i64 sv, i64 n, const double2* __restrict__ in, float4* __restrict__ out) {
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    i64 j = t / sv, cb = t - j * sv;
    double2 a = in[(2 * j) * sv + cb], b = in[(2 * j + 1) * sv + cb];
    out[t] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
  }
}
__global__ void k_f32_to_f64(i64 sv, i64 n, const float4* __restrict__ in, double2* __restrict__ out) {
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < n; t += (i64)gridDim.x * blockDim.x) {
    i64 j = t / sv, cb = t - j * sv;
    float4 v = in[t];
    out[(2 * j) * sv + cb] = make_double2(v.x, v.y);
    out[(2 * j + 1) * sv + cb] = make_double2(v.z, v.w);
  }
}

qxd_status f64_to_f32(qxd_lattice* lat, const double2* in, float4* out, i64 nplanes_sites) {
  k_f64_to_f32<<<grid_cap(nplanes_sites, 256), 256, 0, lat->stream>>>(lat->sv, nplanes_sites, in, out);
  QXD_CHECK_LAUNCH(lat, "k_f64_to_f32");
  return QXD_OK;
}
qxd_status f32_to_f64(qxd_lattice* lat, const float4* in, double2* out, i64 nplanes_sites) {
  k_f32_to_f64<<<grid_cap(nplanes_sites, 256), 256, 0, lat->stream>>>(lat->sv, nplanes_sites, in, out);
  QXD_CHECK_LAUNCH(lat, "k_f32_to_f64");
  return QXD_OK;
}

// One parity of FP32 spinor [6][sv] float4 <-> 16-bit [6][sv] uint2 with a per-site scale.
template <class FMT>
__global__ void k_f32_to_n16(i64 sv, i64 Vh, const float4* __restrict__ in, uint2* __restrict__ out,
                             float* __restrict__ nrm) {
  for (i64 cb = blockIdx.x * (i64)blockDim.x + threadIdx.x; cb < Vh; cb += (i64)gridDim.x * blockDim.x) {
    float4 v[6];
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      v[j] = in[j * sv + cb];
      m = fmaxf(m, fmaxf(fmaxf(fabsf(v[j].x), fabsf(v[j].y)), fmaxf(fabsf(v[j].z), fabsf(v[j].w))));
    }
    float inv = m > 0.f ? 1.f / m : 0.f;
    nrm[cb] = m;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      uint2 o;
      o.x = FMT::pack(v[j].x * inv, v[j].y * inv);
      o.y = FMT::pack(v[j].z * inv, v[j].w * inv);
      out[j * sv + cb] = o;
    }
  }
}
template <class FMT>
__global__ void k_n16_to_f32(i64 sv, i64 Vh, const uint2* __restrict__ in, const float* __restrict__ nrm,
                             float4* __restrict__ out) {
  for (i64 cb = blockIdx.x * (i64)blockDim.x + threadIdx.x; cb < Vh; cb += (i64)gridDim.x * blockDim.x) {
    float n = nrm[cb];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      uint2 v = in[j * sv + cb];
      out[j * sv + cb] = make_float4(n * FMT::lo(v.x), n * FMT::hi(v.x), n * FMT::lo(v.y), n * FMT::hi(v.y));
    }
  }
}

qxd_status f32_to_n16(qxd_lattice* lat, const float4* in, uint2* out, float* nrm, int bf16) {
  if (bf16)
    k_f32_to_n16<B16><<<grid_cap(lat->Vh, 256), 256, 0, lat->stream>>>(lat->sv, lat->Vh, in, out, nrm);
  else
    k_f32_to_n16<H16><<<grid_cap(lat->Vh, 256), 256, 0, lat->stream>>>(lat->sv, lat->Vh, in, out, nrm);
  QXD_CHECK_LAUNCH(lat, "k_f32_to_n16");
  return QXD_OK;
}
qxd_status n16_to_f32(qxd_lattice* lat, const uint2* in, const float* nrm, float4* out, int bf16) {
  if (bf16)
    k_n16_to_f32<B16><<<grid_cap(lat->Vh, 256), 256, 0, lat->stream>>>(lat->sv, lat->Vh, in, nrm, out);
  else
    k_n16_to_f32<H16><<<grid_cap(lat->Vh, 256), 256, 0, lat->stream>>>(lat->sv, lat->Vh, in, nrm, out);
  QXD_CHECK_LAUNCH(lat, "k_n16_to_f32");
  return QXD_OK;
}

}  // namespace qxd
