// C ABI of libqxd (declared in include/qxd.h): argument checks, host/device staging, lattice
// lifetime, work buffers and kernel timing.
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "qxd_internal.cuh"
#include "trace.cuh"

namespace qxd {
qxd_status apply_dhat_prec(qxd_lattice* lat, int prec, const double2* in64, double2* out64, int dag);
qxd_status apply_D_prec(qxd_lattice* lat, int prec, const double2* in64, double2* out64);
}  // namespace qxd

using namespace qxd;

static std::string g_create_error;

enum { AS_IN = 24, AS_OUT = 25, AS_BND_IN = 26, AS_BND_OUT = 27 };

namespace qxd {

qxd_status fail(qxd_lattice* lat, qxd_status st, const std::string& msg) {
  if (lat)
    lat->err = msg;
  else
    g_create_error = msg;
  return st;
}

qxd_status cuda_fail(qxd_lattice* lat, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(lat, e == cudaErrorMemoryAllocation ? QXD_ENOMEM : QXD_ECUDA, m);
}

qxd_status check_device_vector(qxd_lattice* lat, const void* p, size_t align, const char* what) {
  if ((uintptr_t)p % align != 0)
    return fail(lat, QXD_EINVAL, std::string(what) + ": pointer not aligned to " + std::to_string(align) + " bytes");
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // the failed query records a (non-sticky) error: clear it
    return fail(lat, QXD_EINVAL, std::string(what) + ": not a CUDA pointer");
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(lat, QXD_EINVAL, std::string(what) + ": not device memory");
  return QXD_OK;
}

// Guard words: every lattice field and work buffer is allocated GUARD_BYTES longer, and that
// tail is filled with GUARD_FILL.  qxd_check_guards counts tail bytes that changed, so a kernel
// writing past the end of a buffer shows up in the tests without a memory checker.  The guard
// addresses live here, keyed by lattice, one per field and one per work slot.
constexpr size_t GUARD_BYTES = 256;
constexpr unsigned char GUARD_FILL = 0xA5;
struct GuardSet {
  std::vector<unsigned char*> fields;
  unsigned char* work[QXD_WORK_SLOTS] = {};
};
static std::mutex g_guard_mu;
static std::unordered_map<const qxd_lattice*, GuardSet> g_guards;

// cudaMalloc of bytes plus the guard, zeroed, guard filled; slot < 0 registers a field
static qxd_status guarded_malloc(qxd_lattice* lat, void** p, size_t bytes, int slot) {
  QXD_CUDA(lat, cudaMalloc(p, bytes + GUARD_BYTES));
  unsigned char* tail = (unsigned char*)*p + bytes;
  QXD_CUDA(lat, cudaMemsetAsync(*p, 0, bytes, lat->stream));
  QXD_CUDA(lat, cudaMemsetAsync(tail, GUARD_FILL, GUARD_BYTES, lat->stream));
  std::lock_guard<std::mutex> lk(g_guard_mu);
  GuardSet& gs = g_guards[lat];
  if (slot < 0)
    gs.fields.push_back(tail);
  else
    gs.work[slot] = tail;
  return QXD_OK;
}

static void guards_forget(const qxd_lattice* lat) {
  std::lock_guard<std::mutex> lk(g_guard_mu);
  g_guards.erase(lat);
}

qxd_status ensure_work(qxd_lattice* lat, int slot, size_t bytes, void** out) {
  if (slot < 0 || slot >= QXD_WORK_SLOTS) return fail(lat, QXD_EINVAL, "bad work slot");
  if (lat->work_bytes[slot] < bytes) {
    if (lat->work[slot]) {
      QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
      cudaFree(lat->work[slot]);
      lat->work[slot] = nullptr;
      lat->work_bytes[slot] = 0;
      std::lock_guard<std::mutex> lk(g_guard_mu);
      g_guards[lat].work[slot] = nullptr;
    }
    const qxd_status st = guarded_malloc(lat, &lat->work[slot], bytes, slot);
    if (st != QXD_OK) return st;
    lat->work_bytes[slot] = bytes;
  }
  *out = lat->work[slot];
  return QXD_OK;
}

void prof_begin(qxd_lattice* lat, int kind, double bytes) {
  if (!lat->profiling) return;
  size_t need = 2 * (size_t)(lat->ev_used + 1);
  while (lat->ev_pool.size() < need) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      lat->profiling = false;
      return;
    }
    lat->ev_pool.push_back(e);
  }
  if ((int)lat->ev_kind.size() < lat->ev_used + 1) {
    lat->ev_kind.resize(lat->ev_used + 1);
    lat->ev_bytes.resize(lat->ev_used + 1);
  }
  lat->ev_kind[lat->ev_used] = kind;
  lat->ev_bytes[lat->ev_used] = bytes;
  cudaEventRecord(lat->ev_pool[2 * lat->ev_used], lat->stream);
}

void prof_end(qxd_lattice* lat) {
  if (!lat->profiling) return;
  cudaEventRecord(lat->ev_pool[2 * lat->ev_used + 1], lat->stream);
  lat->ev_used++;
}

void prof_set_last_bytes(qxd_lattice* lat, double bytes) {
  if (lat->profiling && lat->ev_used > 0) lat->ev_bytes[lat->ev_used - 1] = bytes;
}

static qxd_status prof_flush(qxd_lattice* lat) {
  if (lat->ev_used == 0) return QXD_OK;
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  for (int i = 0; i < lat->ev_used; ++i) {
    float ms = 0.f;
    QXD_CUDA(lat, cudaEventElapsedTime(&ms, lat->ev_pool[2 * i], lat->ev_pool[2 * i + 1]));
    int k = lat->ev_kind[i];
    lat->kcount[k] += 1;
    lat->kms[k] += ms;
    lat->kbytes[k] += lat->ev_bytes[i];
  }
  lat->ev_used = 0;
  return QXD_OK;
}

qxd_status ensure_stage(qxd_lattice* lat, size_t bytes) {
  void* p;
  qxd_status st = ensure_work(lat, AS_BND_IN, bytes, &p);
  lat->stage = p;
  lat->stage_bytes = bytes;
  return st;
}

}  // namespace qxd

#define CHECK_LAT(lat) \
  if (!(lat)) return QXD_EINVAL

#define TRY(x)                   \
  do {                           \
    qxd_status _s = (x);         \
    if (_s != QXD_OK) return _s; \
  } while (0)

template <typename T>
static qxd_status alloc(qxd_lattice* lat, T** p, size_t bytes) {
  return guarded_malloc(lat, (void**)p, bytes, -1);
}

namespace qxd {
qxd_status sap_check(qxd_lattice* lat, const int b[4]);  // csrc/sap.cu
bool dfl_ready(const qxd_lattice* lat);                  // csrc/dfl.cu
bool mg_ready(const qxd_lattice* lat);                   // csrc/mg.cu

// The caller's params as the current version.  Version 3 ended at `fallback`; version 4 appended
// use_x0 and restart_f32, which a version-3 caller gets off.
qxd_status params_current(qxd_lattice* lat, const qxd_solve_params* p, qxd_solve_params* q) {
  size_t have;
  if (p->version == QXD_PARAMS_VERSION)
    have = sizeof(*q);
  else if (p->version == 4)
    have = offsetof(qxd_solve_params, sap_block);
  else if (p->version == 3)
    have = offsetof(qxd_solve_params, use_x0);
  else
    return fail(lat, QXD_EINVAL, "qxd_solve_params version mismatch");
  qxd_default_params(q);
  std::memcpy(q, p, have);
  if (p->version == 3) {  // version 3 had no initial guess and no FP32 restart
    q->use_x0 = 0;
    q->restart_f32 = 0;
  }
  q->version = QXD_PARAMS_VERSION;
  return QXD_OK;
}
}  // namespace qxd

extern "C" {

void qxd_default_params(qxd_solve_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->version = QXD_PARAMS_VERSION;
  p->solver = QXD_SOLVER_MP_CG_EO;
  p->tol = 1e-10;
  p->maxiter = 100000;
  p->inner_prec = QXD_F32;
  p->inner_tol = 1e-5;
  p->reliable_delta = 0.1;
  p->max_outer = 20;
  p->on_device = 1;
  p->check_every = 1;
  p->gcr_restart = 16;
  p->gcr_reorth = 1;
  p->fallback = -1;
  p->net = nullptr;
  p->use_x0 = 0;
  p->restart_f32 = 1;
  for (int mu = 0; mu < 4; ++mu) p->sap_block[mu] = 4;
  p->sap_ncy = 2;
  p->sap_nmr = 4;
}

qxd_status qxd_destroy_lattice(qxd_lattice* lat) {
  QXD_TRACE();
  if (!lat) return QXD_OK;
  if (lat->stream) cudaStreamSynchronize(lat->stream);
  if (lat->batch && lat->batch_release) lat->batch_release(lat->batch);
  if (lat->mg && lat->mg_release) lat->mg_release(lat->mg);
  if (lat->dfl && lat->dfl_release) lat->dfl_release(lat->dfl);
  void* bufs[] = {lat->U,    lat->A,     lat->W64,   lat->W32,   lat->W16,   lat->WB16,  lat->C64,
                  lat->Ci64, lat->C32,   lat->Ci32,  lat->C16,   lat->Ci16,  lat->C16n,  lat->Ci16n,
                  lat->CB16, lat->CiB16, lat->CB16n, lat->CiB16n, lat->red,  lat->ticket, lat->scal};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int i = 0; i < QXD_WORK_SLOTS; ++i)
    if (lat->work[i]) cudaFree(lat->work[i]);
  void* mr[] = {lat->mr_red, lat->mr_ticket, lat->mr_scal};
  for (void* b : mr)
    if (b) cudaFree(b);
  if (lat->mr_hscal) cudaFreeHost(lat->mr_hscal);
  if (lat->hscal) cudaFreeHost(lat->hscal);
  for (cudaEvent_t e : lat->ev_pool) cudaEventDestroy(e);
  guards_forget(lat);
  delete lat;
  return QXD_OK;
}

qxd_status qxd_check_guards(qxd_lattice* lat, int64_t* bad) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (!bad) return fail(lat, QXD_EINVAL, "null argument");
  std::vector<unsigned char*> tails;
  {
    std::lock_guard<std::mutex> lk(g_guard_mu);
    auto it = g_guards.find(lat);
    if (it != g_guards.end()) {
      tails = it->second.fields;
      for (unsigned char* t : it->second.work)
        if (t) tails.push_back(t);
    }
  }
  std::vector<unsigned char> host(GUARD_BYTES * tails.size());
  for (size_t i = 0; i < tails.size(); ++i)
    QXD_CUDA(lat, cudaMemcpyAsync(host.data() + i * GUARD_BYTES, tails[i], GUARD_BYTES, cudaMemcpyDeviceToHost,
                                  lat->stream));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  int64_t n = 0;
  for (unsigned char c : host) n += c != GUARD_FILL;
  *bad = n;
  if (n) {
    char m[96];
    std::snprintf(m, sizeof(m), "%lld guard bytes overwritten", (long long)n);
    lat->err = m;
  }
  return QXD_OK;
}

qxd_status qxd_create_lattice(const int L[4], int tbc, int cstar, int order, void* cuda_stream, qxd_lattice** out) {
  QXD_TRACE();
  if (!out || !L) return fail(nullptr, QXD_EINVAL, "null argument");
  *out = nullptr;
  for (int mu = 0; mu < 4; ++mu)
    if (L[mu] < 2 || (L[mu] & 1)) return fail(nullptr, QXD_EINVAL, "every extent must be even and >= 2");
  if (tbc != QXD_BC_PERIODIC && tbc != QXD_BC_ANTIPERIODIC) return fail(nullptr, QXD_EINVAL, "bad tbc");
  if (cstar != 0 && cstar != 1) return fail(nullptr, QXD_EINVAL, "cstar must be 0 or 1");
  if (order != QXD_ORDER_LEXI && order != QXD_ORDER_IPT) return fail(nullptr, QXD_EINVAL, "bad order");
  qxd_lattice* lat = new qxd_lattice();
  lat->stream = (cudaStream_t)cuda_stream;
  lat->tbc = tbc;
  lat->cstar = cstar;
  lat->order = order;
  for (int mu = 0; mu < 4; ++mu) {
    lat->Lphys[mu] = L[mu];
    lat->g.L[mu] = L[mu];
  }
  if (cstar) lat->g.L[1] = 2 * L[1];
  lat->g.shift = cstar ? L[1] : 0;
  lat->g.anti = tbc == QXD_BC_ANTIPERIODIC;
  lat->V = (i64)lat->g.L[0] * lat->g.L[1] * lat->g.L[2] * lat->g.L[3];
  lat->Vphys = (i64)L[0] * L[1] * L[2] * L[3];
  lat->Vh = lat->V / 2;
  lat->sv = (lat->Vh + 63) / 64 * 64;
  lat->g.Vh = lat->Vh;
  lat->g.sv = lat->sv;
  if (lat->V >= (i64)1 << 31) {
    delete lat;
    return fail(nullptr, QXD_EINVAL, "volume must be below 2^31 sites");
  }
  for (int mu = 0; mu < 4; ++mu) lat->g.B[mu] = lat->g.L[mu];  // IPT order: one cache block
  lat->g.dL1 = make_fastdiv((uint32_t)lat->g.L[1]);
  lat->g.dL2 = make_fastdiv((uint32_t)lat->g.L[2]);
  lat->g.dL3 = make_fastdiv((uint32_t)lat->g.L[3]);
  cudaGetDevice(&lat->device);
  const i64 sv = lat->sv;
  qxd_status st = QXD_OK;
#define ALLOC(p, bytes)                            \
  if ((st = alloc(lat, &lat->p, (bytes))) != QXD_OK) { \
    g_create_error = lat->err;                     \
    qxd_destroy_lattice(lat);                      \
    return st;                                     \
  }
  ALLOC(U, sizeof(float4) * 72 * sv);
  ALLOC(A, sizeof(double) * 8 * sv);
  ALLOC(W64, sizeof(double2) * 72 * sv);
  ALLOC(W32, sizeof(float2) * 72 * sv);
  ALLOC(W16, sizeof(uint32_t) * 72 * sv);
  ALLOC(WB16, sizeof(uint32_t) * 72 * sv);
  ALLOC(C64, sizeof(double2) * 72 * sv);
  ALLOC(Ci64, sizeof(double2) * 72 * sv);
  ALLOC(C32, sizeof(float4) * 36 * sv);
  ALLOC(Ci32, sizeof(float4) * 36 * sv);
  ALLOC(C16, sizeof(uint2) * 36 * sv);
  ALLOC(Ci16, sizeof(uint2) * 36 * sv);
  ALLOC(C16n, sizeof(float) * 4 * sv);
  ALLOC(Ci16n, sizeof(float) * 4 * sv);
  ALLOC(CB16, sizeof(uint2) * 36 * sv);
  ALLOC(CiB16, sizeof(uint2) * 36 * sv);
  ALLOC(CB16n, sizeof(float) * 4 * sv);
  ALLOC(CiB16n, sizeof(float) * 4 * sv);
  lat->red_blocks = 152 * 8;
  ALLOC(red, sizeof(double) * 4 * lat->red_blocks);  // partial sums: up to 4 values per reduction block
  ALLOC(ticket, sizeof(unsigned int) * 4);
  ALLOC(scal, sizeof(double) * SC_N);
#undef ALLOC
  if (cudaMallocHost((void**)&lat->hscal, sizeof(double) * SC_N) != cudaSuccess) {
    g_create_error = "cudaMallocHost failed";
    qxd_destroy_lattice(lat);
    return QXD_ENOMEM;
  }
  if (cudaStreamSynchronize(lat->stream) != cudaSuccess) {
    g_create_error = "stream synchronisation failed after allocation";
    qxd_destroy_lattice(lat);
    return QXD_ECUDA;
  }
  *out = lat;
  return QXD_OK;
}

qxd_status qxd_load_gauge(qxd_lattice* lat, const double* su3, const double* a_u1, double q, int on_device) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (!su3) return fail(lat, QXD_EINVAL, "su3 is null");
  const i64 Vp = lat->Vphys;
  const size_t ub = sizeof(double2) * 36 * Vp, ab = sizeof(double) * 4 * Vp;
  lat->q = q;
  const double2* dsu3 = (const double2*)su3;
  const double* da = a_u1;
  if (!on_device) {
    void* p;
    TRY(ensure_work(lat, AS_BND_IN, ub, &p));
    QXD_CUDA(lat, cudaMemcpyAsync(p, su3, ub, cudaMemcpyHostToDevice, lat->stream));
    dsu3 = (const double2*)p;
    if (a_u1) {
      TRY(ensure_work(lat, AS_BND_OUT, ab, &p));
      QXD_CUDA(lat, cudaMemcpyAsync(p, a_u1, ab, cudaMemcpyHostToDevice, lat->stream));
      da = (const double*)p;
    }
  }
  TRY(ingest_gauge(lat, dsu3, da));
  TRY(convert_links_low(lat));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  lat->have_gauge = true;
  lat->have_clover = false;
  lat->epoch++;
  return QXD_OK;
}

qxd_status qxd_update_links(qxd_lattice* lat, int64_t n, const int64_t* idx, const double* su3, const double* a_u1,
                            int on_device) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (!lat->have_gauge) return fail(lat, QXD_ESTATE, "update_links before load_gauge");
  if (n < 0) return fail(lat, QXD_EINVAL, "n must be >= 0");
  if (n == 0) return QXD_OK;
  if (!idx || !su3) return fail(lat, QXD_EINVAL, "idx and su3 must not be null");
  const Geom& g = lat->g;
  const int64_t* d_idx = idx;
  const double2* d_su3 = (const double2*)su3;
  const double* d_a = a_u1;
  if (!on_device) {  // stage the host arrays: idx, then su3, then the angles
    unsigned char* st;
    TRY(ensure_work(lat, 49, (size_t)n * (sizeof(int64_t) + sizeof(double2) * 9 + sizeof(double)), (void**)&st));
    QXD_CUDA(lat, cudaMemcpyAsync(st, idx, sizeof(int64_t) * n, cudaMemcpyHostToDevice, lat->stream));
    QXD_CUDA(lat, cudaMemcpyAsync(st + sizeof(int64_t) * n, su3, sizeof(double2) * 9 * n, cudaMemcpyHostToDevice,
                                  lat->stream));
    d_idx = (const int64_t*)st;
    d_su3 = (const double2*)(st + sizeof(int64_t) * n);
    if (a_u1) {
      double* da = (double*)(st + (sizeof(int64_t) + sizeof(double2) * 9) * n);
      QXD_CUDA(lat, cudaMemcpyAsync(da, a_u1, sizeof(double) * n, cudaMemcpyHostToDevice, lat->stream));
      d_a = da;
    }
  }
  // slot 48: the clover-site mask [2 Vh] bytes, then the list count and the bad-index flag
  const i64 nsite = 2 * g.Vh;
  const size_t mask_bytes = ((size_t)nsite + 255) / 256 * 256;
  unsigned char* mask;
  TRY(ensure_work(lat, 48, mask_bytes + 2 * sizeof(int), (void**)&mask));
  unsigned int* count = (unsigned int*)(mask + mask_bytes);
  int* bad = (int*)(count + 1);
  QXD_CUDA(lat, cudaMemsetAsync(mask, 0, mask_bytes + 2 * sizeof(int), lat->stream));
  lat->epoch++;
  TRY(update_links(lat, n, d_idx, d_su3, d_a, mask, bad));
  int hbad[2] = {0, 0};
  if (lat->have_clover) {
    // slot 50: the site list [2 Vh] and the field strengths of the listed sites (60 doubles each)
    uint32_t* list;
    TRY(ensure_work(lat, 50, sizeof(uint32_t) * nsite, (void**)&list));
    TRY(compact_mask(lat, mask, list, count));
    QXD_CUDA(lat, cudaMemcpyAsync(hbad, count, 2 * sizeof(int), cudaMemcpyDeviceToHost, lat->stream));
    QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
    const i64 nl = (i64)(unsigned int)hbad[0];
    if (hbad[1]) {
      lat->have_clover = false;  // stale at the updated links: build_clover must run before the next apply
      return fail(lat, QXD_EINVAL, "update_links: a link index is outside 0 .. 4 V - 1 (skipped)");
    }
    if (nl > nsite / 4) {
      // most of the lattice changed: the full build (shared plaquette half-products) is cheaper
      lat->have_clover = false;
      TRY(clover_build(lat));
      lat->have_clover = true;
      return QXD_OK;
    }
    double* Fc;
    TRY(ensure_work(lat, 51, sizeof(double) * 60 * (size_t)(nl > 0 ? nl : 1), (void**)&Fc));
    int* sbad = bad;  // reused as the singular-block flag
    QXD_CUDA(lat, cudaMemsetAsync(sbad, 0, sizeof(int), lat->stream));
    TRY(clover_rebuild_sites(lat, list, nl, Fc, sbad));
    QXD_CUDA(lat, cudaMemcpyAsync(hbad + 1, sbad, sizeof(int), cudaMemcpyDeviceToHost, lat->stream));
    QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
    if (hbad[1]) {
      lat->have_clover = false;
      return fail(lat, QXD_ESINGULAR, "update_links: a rebuilt clover block on an odd site is not invertible");
    }
    return QXD_OK;
  }
  QXD_CUDA(lat, cudaMemcpyAsync(hbad + 1, bad, sizeof(int), cudaMemcpyDeviceToHost, lat->stream));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  if (hbad[1]) return fail(lat, QXD_EINVAL, "update_links: a link index is outside 0 .. 4 V - 1 (skipped)");
  return QXD_OK;
}

qxd_status qxd_set_ipt_blocks(qxd_lattice* lat, const int B[4]) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (!B) return fail(lat, QXD_EINVAL, "B is null");
  if (lat->order != QXD_ORDER_IPT) return fail(lat, QXD_EINVAL, "cache blocks need QXD_ORDER_IPT");
  for (int mu = 0; mu < 4; ++mu) {
    // the blocks must tile the physical lattice (gauge input) and the device lattice (doubled in x for C*)
    if (B[mu] < 1 || lat->Lphys[mu] % B[mu] != 0 || lat->g.L[mu] % B[mu] != 0)
      return fail(lat, QXD_EINVAL, "each block extent must divide the lattice extent");
  }
  for (int mu = 0; mu < 4; ++mu) lat->g.B[mu] = B[mu];
  return QXD_OK;
}

qxd_status qxd_load_gauge_openqxd(qxd_lattice* lat, const double* u8, const double* a8, double q, int on_device) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (!u8) return fail(lat, QXD_EINVAL, "u8 is null");
  if (lat->order != QXD_ORDER_IPT) return fail(lat, QXD_EINVAL, "the openQxD gauge format needs QXD_ORDER_IPT");
  const i64 V = lat->V;
  const size_t ub = sizeof(double2) * 36 * V, ab = sizeof(double) * 4 * V;  // V/2 odd sites x 8 links
  lat->q = q;
  const double2* du = (const double2*)u8;
  const double* da = a8;
  if (!on_device) {
    void* p;
    TRY(ensure_work(lat, AS_BND_IN, ub, &p));
    QXD_CUDA(lat, cudaMemcpyAsync(p, u8, ub, cudaMemcpyHostToDevice, lat->stream));
    du = (const double2*)p;
    if (a8) {
      TRY(ensure_work(lat, AS_BND_OUT, ab, &p));
      QXD_CUDA(lat, cudaMemcpyAsync(p, a8, ab, cudaMemcpyHostToDevice, lat->stream));
      da = (const double*)p;
    }
  }
  TRY(ingest_gauge_openqxd(lat, du, da));
  TRY(convert_links_low(lat));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  lat->have_gauge = true;
  lat->have_clover = false;
  lat->epoch++;
  return QXD_OK;
}

qxd_status qxd_build_clover(qxd_lattice* lat, double m0, double csw, double csw_qed) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (!lat->have_gauge) return fail(lat, QXD_ESTATE, "build_clover before load_gauge");
  lat->m0 = m0;
  lat->csw = csw;
  lat->csw_qed = csw_qed;
  lat->have_clover = false;
  lat->epoch++;
  TRY(clover_build(lat));
  lat->have_clover = true;
  return QXD_OK;
}

qxd_status qxd_get_clover(qxd_lattice* lat, double* out, int on_device) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (!out) return fail(lat, QXD_EINVAL, "out is null");
  if (!lat->have_clover) return fail(lat, QXD_ESTATE, "get_clover before build_clover");
  const size_t bytes = sizeof(double) * 72 * lat->V;
  if (on_device) return clover_export(lat, out);
  void* p;
  TRY(ensure_work(lat, AS_BND_OUT, bytes, &p));
  TRY(clover_export(lat, (double*)p));
  QXD_CUDA(lat, cudaMemcpyAsync(out, p, bytes, cudaMemcpyDeviceToHost, lat->stream));
  QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  return QXD_OK;
}

qxd_status qxd_apply_D(qxd_lattice* lat, double* out, const double* in, int prec, int nrhs, int on_device) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (!out || !in) return fail(lat, QXD_EINVAL, "null field pointer");
  if (nrhs <= 0) return fail(lat, QXD_EINVAL, "nrhs must be positive");
  if (prec < QXD_F64 || prec > QXD_BF16N) return fail(lat, QXD_EINVAL, "bad precision");
  if (!lat->have_clover) return fail(lat, QXD_ESTATE, "apply_D before build_clover");
  const i64 sv = lat->sv;
  const size_t fb = sizeof(double2) * 24 * sv, vb = sizeof(double) * 24 * lat->V;
  double2 *fin, *fout;
  void *bi, *bo;
  TRY(ensure_work(lat, AS_IN, fb, (void**)&fin));
  TRY(ensure_work(lat, AS_OUT, fb, (void**)&fout));
  if (!on_device) {
    TRY(ensure_work(lat, AS_BND_IN, vb, &bi));
    TRY(ensure_work(lat, AS_BND_OUT, vb, &bo));
  }
  if (prec == QXD_F32 && nrhs > 1) {
    // multi-RHS FP32 path: one link/clover load per site serves every right-hand side
    float4 *mi, *mo;
    TRY(ensure_work(lat, 37, sizeof(float4) * 12 * sv * nrhs, (void**)&mi));
    TRY(ensure_work(lat, 38, sizeof(float4) * 12 * sv * nrhs, (void**)&mo));
    for (int r = 0; r < nrhs; ++r) {
      const double* src = in + (i64)r * 24 * lat->V;
      if (!on_device) {
        QXD_CUDA(lat, cudaMemcpyAsync(bi, src, vb, cudaMemcpyHostToDevice, lat->stream));
        src = (const double*)bi;
      }
      TRY(pack_spinor64(lat, (const double2*)src, fin, 0));
      TRY(f64_to_f32(lat, fin, mi + (i64)r * 12 * sv, 12 * sv));
    }
    const i64 rs = 12 * sv;
    TRY(hop32_mrhs(lat, 0, EPI_DFULL, 0, mi + 6 * sv, mi, mo, 0.f, nrhs, rs));
    TRY(hop32_mrhs(lat, 1, EPI_DFULL, 0, mi, mi + 6 * sv, mo + 6 * sv, 0.f, nrhs, rs));
    TRY(mrhs_tile_status(lat));
    for (int r = 0; r < nrhs; ++r) {
      double* dst = out + (i64)r * 24 * lat->V;
      TRY(f32_to_f64(lat, mo + (i64)r * 12 * sv, fout, 12 * sv));
      TRY(unpack_spinor64(lat, fout, on_device ? (double2*)dst : (double2*)bo, 0));
      if (!on_device) {
        QXD_CUDA(lat, cudaMemcpyAsync(dst, bo, vb, cudaMemcpyDeviceToHost, lat->stream));
        QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
      }
    }
    return QXD_OK;
  }
  if ((prec == QXD_F16N || prec == QXD_BF16N) && nrhs > 1) {
    // multi-RHS 16-bit path: per parity, the right-hand sides' 16-bit copies (with per-site
    // norms) sit one after another, [rhs][6][sv]; one link/clover tile load serves all of them
    const int bf = prec == QXD_BF16N;
    const i64 h = 6 * sv * nrhs;  // float4 (or uint2) entries of one parity of all RHS
    float4* m32;
    uint2* m16;
    TRY(ensure_work(lat, 37, sizeof(float4) * 2 * h, (void**)&m32));
    TRY(ensure_work(lat, 38, sizeof(uint2) * 2 * h + sizeof(float) * 2 * sv * nrhs, (void**)&m16));
    float* n16 = (float*)(m16 + 2 * h);
    for (int r = 0; r < nrhs; ++r) {
      const double* src = in + (i64)r * 24 * lat->V;
      if (!on_device) {
        QXD_CUDA(lat, cudaMemcpyAsync(bi, src, vb, cudaMemcpyHostToDevice, lat->stream));
        src = (const double*)bi;
      }
      TRY(pack_spinor64(lat, (const double2*)src, fin, 0));
      for (int par = 0; par < 2; ++par) {
        float4* f = m32 + par * h + (i64)r * 6 * sv;
        TRY(f64_to_f32(lat, fin + (i64)par * 12 * sv, f, 6 * sv));
        TRY(f32_to_n16(lat, f, m16 + par * h + (i64)r * 6 * sv, n16 + (par * nrhs + r) * sv, bf));
      }
    }
    for (int par = 0; par < 2; ++par)
      TRY(hop16_mrhs(lat, bf, par, EPI_DFULL, 0, m16 + (1 - par) * h, n16 + (i64)(1 - par) * nrhs * sv,
                     m16 + par * h, n16 + (i64)par * nrhs * sv, nullptr, nullptr, m32 + par * h, 0.f, nrhs));
    for (int r = 0; r < nrhs; ++r) {
      double* dst = out + (i64)r * 24 * lat->V;
      for (int par = 0; par < 2; ++par)
        TRY(f32_to_f64(lat, m32 + par * h + (i64)r * 6 * sv, fout + (i64)par * 12 * sv, 6 * sv));
      TRY(unpack_spinor64(lat, fout, on_device ? (double2*)dst : (double2*)bo, 0));
      if (!on_device) {
        QXD_CUDA(lat, cudaMemcpyAsync(dst, bo, vb, cudaMemcpyDeviceToHost, lat->stream));
        QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
      }
    }
    return QXD_OK;
  }
  for (int r = 0; r < nrhs; ++r) {
    const double* src = in + (i64)r * 24 * lat->V;
    double* dst = out + (i64)r * 24 * lat->V;
    if (!on_device) {
      QXD_CUDA(lat, cudaMemcpyAsync(bi, src, vb, cudaMemcpyHostToDevice, lat->stream));
      src = (const double*)bi;
    }
    TRY(pack_spinor64(lat, (const double2*)src, fin, 0));
    TRY(apply_D_prec(lat, prec, fin, fout));
    TRY(unpack_spinor64(lat, fout, on_device ? (double2*)dst : (double2*)bo, 0));
    if (!on_device) QXD_CUDA(lat, cudaMemcpyAsync(dst, bo, vb, cudaMemcpyDeviceToHost, lat->stream));
  }
  if (!on_device) QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  return QXD_OK;
}

qxd_status qxd_apply_Dhat_eo(qxd_lattice* lat, double* out_e, const double* in_e, int prec, int dagger,
                             int on_device) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (!out_e || !in_e) return fail(lat, QXD_EINVAL, "null field pointer");
  if (prec < QXD_F64 || prec > QXD_BF16N) return fail(lat, QXD_EINVAL, "bad precision");
  if (!lat->have_clover) return fail(lat, QXD_ESTATE, "apply_Dhat_eo before build_clover");
  const i64 sv = lat->sv;
  const size_t hb = sizeof(double2) * 12 * sv, vb = sizeof(double) * 24 * lat->Vh;
  double2 *fin, *fout;
  TRY(ensure_work(lat, AS_IN, sizeof(double2) * 24 * sv, (void**)&fin));
  TRY(ensure_work(lat, AS_OUT, sizeof(double2) * 24 * sv, (void**)&fout));
  (void)hb;
  const double* src = in_e;
  void *bi = nullptr, *bo = nullptr;
  if (!on_device) {
    TRY(ensure_work(lat, AS_BND_IN, vb, &bi));
    TRY(ensure_work(lat, AS_BND_OUT, vb, &bo));
    QXD_CUDA(lat, cudaMemcpyAsync(bi, in_e, vb, cudaMemcpyHostToDevice, lat->stream));
    src = (const double*)bi;
  }
  TRY(pack_spinor64(lat, (const double2*)src, fin, 1));
  TRY(apply_dhat_prec(lat, prec, fin, fout, dagger ? 1 : 0));
  TRY(unpack_spinor64(lat, fout, on_device ? (double2*)out_e : (double2*)bo, 1));
  if (!on_device) {
    QXD_CUDA(lat, cudaMemcpyAsync(out_e, bo, vb, cudaMemcpyDeviceToHost, lat->stream));
    QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  }
  return QXD_OK;
}

qxd_status qxd_solve(qxd_lattice* lat, double* x, const double* b, const qxd_solve_params* p, qxd_solve_info* info) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (info) std::memset(info, 0, sizeof(*info));
  if (!x || !b || !p) return fail(lat, QXD_EINVAL, "null argument");
  qxd_solve_params pv;
  TRY(params_current(lat, p, &pv));
  p = &pv;
  if (p->solver != QXD_SOLVER_CG_EO && p->solver != QXD_SOLVER_MP_CG_EO && p->solver != QXD_SOLVER_MP_BICGSTAB_EO &&
      p->solver != QXD_SOLVER_MP_FGCR_NET && p->solver != QXD_SOLVER_MP_SAP_GCR && p->solver != QXD_SOLVER_MP_CGNR &&
      p->solver != QXD_SOLVER_MP_DFL_SAP_GCR && p->solver != QXD_SOLVER_MP_MG_GCR)
    return fail(lat, QXD_EINVAL, "bad solver");
  if (p->solver == QXD_SOLVER_MP_DFL_SAP_GCR && !dfl_ready(lat))
    return fail(lat, QXD_ESTATE, "DFL_SAP_GCR needs a deflation subspace set up on the current field (qxd_dfl_setup)");
  if (p->solver == QXD_SOLVER_MP_MG_GCR && !mg_ready(lat))
    return fail(lat, QXD_ESTATE,
                "MG_GCR needs a multigrid set up on the current deflation subspace (qxd_dfl_setup, then qxd_mg_setup)");
  if (p->solver == QXD_SOLVER_MP_SAP_GCR || p->solver == QXD_SOLVER_MP_DFL_SAP_GCR || p->solver == QXD_SOLVER_MP_MG_GCR) {
    TRY(sap_check(lat, p->sap_block));
    if (p->sap_ncy < 1 || p->sap_nmr < 1) return fail(lat, QXD_EINVAL, "sap_ncy and sap_nmr must be >= 1");
  }
  if (p->fallback != -1 && p->fallback != QXD_SOLVER_CG_EO && p->fallback != QXD_SOLVER_MP_CG_EO &&
      p->fallback != QXD_SOLVER_MP_BICGSTAB_EO)
    return fail(lat, QXD_EINVAL, "fallback must be -1, CG_EO, MP_CG_EO or MP_BICGSTAB_EO");
  if (p->use_x0 != 0 && p->use_x0 != 1) return fail(lat, QXD_EINVAL, "use_x0 must be 0 or 1");
  if (p->restart_f32 != 0 && p->restart_f32 != 1) return fail(lat, QXD_EINVAL, "restart_f32 must be 0 or 1");
  const bool fgcr = p->solver == QXD_SOLVER_MP_FGCR_NET || p->solver == QXD_SOLVER_MP_SAP_GCR ||
                    p->solver == QXD_SOLVER_MP_DFL_SAP_GCR || p->solver == QXD_SOLVER_MP_MG_GCR;
  if (fgcr && (p->gcr_reorth < 1 || p->gcr_reorth > 2)) return fail(lat, QXD_EINVAL, "gcr_reorth must be 1 or 2");
  if (fgcr && (p->gcr_restart < 1 || p->gcr_restart > 32)) return fail(lat, QXD_EINVAL, "gcr_restart must be 1..32");
  if (!(p->tol > 0) || p->maxiter <= 0) return fail(lat, QXD_EINVAL, "tol must be > 0 and maxiter > 0");
  if (p->solver != QXD_SOLVER_CG_EO && (p->inner_prec < QXD_F32 || p->inner_prec > QXD_BF16N))
    return fail(lat, QXD_EINVAL, "inner_prec must be F32, F16N or BF16N");
  if (!lat->have_clover) return fail(lat, QXD_ESTATE, "solve before build_clover");
  const i64 sv = lat->sv;
  const size_t fb = sizeof(double2) * 24 * sv, vb = sizeof(double) * 24 * lat->V;
  double2 *fb_in, *fx;
  TRY(ensure_work(lat, AS_IN, fb, (void**)&fb_in));
  TRY(ensure_work(lat, AS_OUT, fb, (void**)&fx));
  const double* src = b;
  void *bi = nullptr, *bo = nullptr;
  if (!p->on_device) {
    TRY(ensure_work(lat, AS_BND_IN, vb, &bi));
    TRY(ensure_work(lat, AS_BND_OUT, vb, &bo));
    QXD_CUDA(lat, cudaMemcpyAsync(bi, b, vb, cudaMemcpyHostToDevice, lat->stream));
    src = (const double*)bi;
  }
  TRY(pack_spinor64(lat, (const double2*)src, fb_in, 0));
  if (p->use_x0) {  // the initial guess, in the same boundary layout as b
    const double* x0 = x;
    if (!p->on_device) {
      QXD_CUDA(lat, cudaMemcpyAsync(bo, x, vb, cudaMemcpyHostToDevice, lat->stream));
      x0 = (const double*)bo;
    }
    TRY(pack_spinor64(lat, (const double2*)x0, fx, 0));
  }
  qxd_status st = solve(lat, fx, fb_in, p, info);
  if (st != QXD_OK && st != QXD_ENOCONV) return st;
  qxd_status st2 = unpack_spinor64(lat, fx, p->on_device ? (double2*)x : (double2*)bo, 0);
  if (st2 != QXD_OK) return st2;
  if (!p->on_device) {
    QXD_CUDA(lat, cudaMemcpyAsync(x, bo, vb, cudaMemcpyDeviceToHost, lat->stream));
    QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
  }
  return st;
}

qxd_status qxd_solve_mrhs(qxd_lattice* lat, double* x, const double* b, int nrhs, const qxd_solve_params* p,
                          qxd_solve_info* info) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (info && nrhs > 0) std::memset(info, 0, sizeof(*info) * nrhs);
  if (!x || !b || !p) return fail(lat, QXD_EINVAL, "null argument");
  if (nrhs <= 0) return fail(lat, QXD_EINVAL, "nrhs must be positive");
  qxd_solve_params pv;
  TRY(params_current(lat, p, &pv));
  p = &pv;
  if (p->use_x0) return fail(lat, QXD_EINVAL, "use_x0 is supported by qxd_solve only");
  if (p->solver != QXD_SOLVER_MP_BICGSTAB_EO ||
      (p->inner_prec != QXD_F32 && p->inner_prec != QXD_F16N && p->inner_prec != QXD_BF16N))
    return fail(lat, QXD_EINVAL, "multi-RHS solve: solver must be MP_BICGSTAB_EO with inner_prec F32, F16N or BF16N");
  if (!(p->tol > 0) || p->maxiter <= 0) return fail(lat, QXD_EINVAL, "tol must be > 0 and maxiter > 0");
  if (!lat->have_clover) return fail(lat, QXD_ESTATE, "solve before build_clover");
  const i64 sv = lat->sv;
  const size_t vb = sizeof(double) * 24 * lat->V;
  double2 *fb, *fx;
  TRY(ensure_work(lat, 37, sizeof(double2) * 24 * sv * nrhs, (void**)&fb));
  TRY(ensure_work(lat, 38, sizeof(double2) * 24 * sv * nrhs, (void**)&fx));
  void *bi = nullptr, *bo = nullptr;
  if (!p->on_device) {
    TRY(ensure_work(lat, AS_BND_IN, vb, &bi));
    TRY(ensure_work(lat, AS_BND_OUT, vb, &bo));
  }
  for (int r = 0; r < nrhs; ++r) {
    const double* src = b + (i64)r * 24 * lat->V;
    if (!p->on_device) {
      QXD_CUDA(lat, cudaMemcpyAsync(bi, src, vb, cudaMemcpyHostToDevice, lat->stream));
      src = (const double*)bi;
    }
    TRY(pack_spinor64(lat, (const double2*)src, fb + (i64)r * 24 * sv, 0));
  }
  qxd_status st = solve_mrhs(lat, fx, fb, nrhs, p, info);
  if (st != QXD_OK && st != QXD_ENOCONV) return st;
  for (int r = 0; r < nrhs; ++r) {
    double* dst = x + (i64)r * 24 * lat->V;
    TRY(unpack_spinor64(lat, fx + (i64)r * 24 * sv, p->on_device ? (double2*)dst : (double2*)bo, 0));
    if (!p->on_device) {
      QXD_CUDA(lat, cudaMemcpyAsync(dst, bo, vb, cudaMemcpyDeviceToHost, lat->stream));
      QXD_CUDA(lat, cudaStreamSynchronize(lat->stream));
    }
  }
  return st;
}

qxd_status qxd_vec_dot(qxd_lattice* lat, const double* a, const double* b, int64_t n, double* re, double* im) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (!re || !im || n < 0 || (n > 0 && (!a || !b))) return fail(lat, QXD_EINVAL, "bad argument");
  if (n == 0) {
    *re = *im = 0.0;
    return QXD_OK;
  }
  TRY(check_device_vector(lat, a, 16, "qxd_vec_dot: a"));
  TRY(check_device_vector(lat, b, 16, "qxd_vec_dot: b"));
  TRY(blas_dot_64(lat, (const double2*)a, (const double2*)b, n, SC_TMP2));
  double v[2];
  TRY(read_scalars(lat, SC_TMP2, 2, v));
  *re = v[0];
  *im = v[1];
  return QXD_OK;
}

qxd_status qxd_vec_norm2(qxd_lattice* lat, const double* a, int64_t n, double* out) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (!out || n < 0 || (n > 0 && !a)) return fail(lat, QXD_EINVAL, "bad argument");
  if (n == 0) {
    *out = 0.0;
    return QXD_OK;
  }
  TRY(check_device_vector(lat, a, 16, "qxd_vec_norm2: a"));
  TRY(blas_norm2_64(lat, (const double2*)a, n, SC_TMP1));
  return read_scalars(lat, SC_TMP1, 1, out);
}

qxd_status qxd_vec_axpy(qxd_lattice* lat, double re, double im, const double* x, double* y, int64_t n) {
  QXD_TRACE();
  CHECK_LAT(lat);
  if (n < 0 || (n > 0 && (!x || !y))) return fail(lat, QXD_EINVAL, "bad argument");
  if (n == 0) return QXD_OK;
  TRY(check_device_vector(lat, x, 16, "qxd_vec_axpy: x"));
  TRY(check_device_vector(lat, y, 16, "qxd_vec_axpy: y"));
  return blas_axpy_64(lat, re, im, (const double2*)x, (double2*)y, n);
}

qxd_status qxd_set_profiling(qxd_lattice* lat, int on) {
  CHECK_LAT(lat);
  TRY(prof_flush(lat));
  lat->profiling = on != 0;
  for (int k = 0; k < KSTAT_N; ++k) {
    lat->kcount[k] = 0;
    lat->kms[k] = 0;
    lat->kbytes[k] = 0;
  }
  return QXD_OK;
}

qxd_status qxd_kernel_stats(qxd_lattice* lat, int which, int64_t* launches, double* ms, double* bytes) {
  CHECK_LAT(lat);
  if (which < 0 || which >= KSTAT_N || !launches || !ms || !bytes) return fail(lat, QXD_EINVAL, "bad argument");
  TRY(prof_flush(lat));
  *launches = lat->kcount[which];
  *ms = lat->kms[which];
  *bytes = lat->kbytes[which];
  return QXD_OK;
}

int64_t qxd_launch_count(const qxd_lattice* lat) { return lat ? lat->launches : 0; }

const char* qxd_last_error(const qxd_lattice* lat) {
  if (!lat) return g_create_error.c_str();
  return lat->err.c_str();
}

}  // extern "C"
