// qxd_vec_dot_noalloc: the deterministic FP64 dot product for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code running inside a framework whose device memory is
// owned by a caching allocator it must not bypass, and latency-critical loops that cannot
// afford the implicit device synchronisation cudaMalloc and cudaFree can cause.  Such a caller
// already owns its input vectors and a 2-double output slot; this entry point needs nothing
// else.
//
// The kernel is the two-level reduction of qxd_vec_dot (block partial sums, the last block to
// finish sums the partials in block order), scheduled in fixed chunks of CHUNK entries per
// block so that the result does not depend on the number of SMs.  Its scratch -- one partial
// (re, im) per block and the ticket counter -- lives in the file-scope array g_scratch below,
// which every GPU that loads the library holds until exit.
#include <mutex>

#include "qxd_internal.cuh"

namespace {

constexpr int THREADS = 256;
constexpr int ITEMS = 16;
constexpr long long CHUNK = (long long)THREADS * ITEMS;                 // entries per block
constexpr int MAX_BLOCKS = (int)(QXD_NOALLOC_MAX_N / CHUNK);           // 4096
constexpr size_t PARTIAL_BYTES = sizeof(double) * 2 * MAX_BLOCKS;      // 64 KiB
constexpr size_t SCRATCH_BYTES = PARTIAL_BYTES + 256;                  // + ticket, padded

static_assert(QXD_NOALLOC_MAX_N % CHUNK == 0, "capacity must be a whole number of chunks");

// Scratch of qxd_vec_dot_noalloc: partials [2][MAX_BLOCKS] doubles, then the ticket counter.
// Host code must not pass g_scratch itself to a kernel (in host code the name is a host-side
// stand-in); it uses the device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum two values over the block; thread 0 returns the totals.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sh[2][THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) {
    sh[0][w] = a;
    sh[1][w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = warp_sum(lane < THREADS / 32 ? sh[0][lane] : 0.0);
    b = warp_sum(lane < THREADS / 32 ? sh[1][lane] : 0.0);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(THREADS) k_dot_noalloc(const double2* __restrict__ a, const double2* __restrict__ b,
                                                        long long n, unsigned char* scratch, double* out) {
  double* partial = reinterpret_cast<double*>(scratch);
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + PARTIAL_BYTES);
  double re = 0.0, im = 0.0;
  const long long base = (long long)blockIdx.x * CHUNK;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    long long i = base + (long long)j * THREADS + threadIdx.x;
    if (i < n) {
      double2 x = a[i], y = b[i];
      re += x.x * y.x + x.y * y.y;  // conj(x) y
      im += x.x * y.y - x.y * y.x;
    }
  }
  block_sum2(re, im);
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = re;
    partial[MAX_BLOCKS + blockIdx.x] = im;
    __threadfence();
    is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double sre = 0.0, sim = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += THREADS) {
    sre += __ldcg(partial + k);
    sim += __ldcg(partial + MAX_BLOCKS + k);
  }
  block_sum2(sre, sim);
  if (threadIdx.x == 0) {
    out[0] = sre;
    out[1] = sim;
    *ticket = 0u;
  }
}

// Device address of g_scratch on the current device, looked up once per device.
qxd_status scratch_address(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return qxd::cuda_fail(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return qxd::fail(nullptr, QXD_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return qxd::cuda_fail(nullptr, e, "cudaGetSymbolAddress(g_scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return QXD_OK;
}

}  // namespace

extern "C" qxd_status qxd_vec_dot_noalloc(const double* a, const double* b, int64_t n, double* out,
                                          void* cuda_stream) {
  if (n < 0 || !out || (n > 0 && (!a || !b))) return qxd::fail(nullptr, QXD_EINVAL, "qxd_vec_dot_noalloc: bad argument");
  if (n > QXD_NOALLOC_MAX_N)
    return qxd::fail(nullptr, QXD_EINVAL,
                     "qxd_vec_dot_noalloc: n exceeds the static scratch capacity of 16777216 complex entries");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the kernel reads a and b as 16-byte complex words and writes out as doubles: refuse host
  // pointers and misaligned views here rather than fault on the GPU
  qxd_status c = qxd::check_device_vector(nullptr, out, 8, "qxd_vec_dot_noalloc: out");
  if (c == QXD_OK && n > 0) c = qxd::check_device_vector(nullptr, a, 16, "qxd_vec_dot_noalloc: a");
  if (c == QXD_OK && n > 0) c = qxd::check_device_vector(nullptr, b, 16, "qxd_vec_dot_noalloc: b");
  if (c != QXD_OK) return c;
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(double), st);
    return e == cudaSuccess ? QXD_OK : qxd::cuda_fail(nullptr, e, "cudaMemsetAsync(out)");
  }
  unsigned char* scratch = nullptr;
  qxd_status s = scratch_address(&scratch);
  if (s != QXD_OK) return s;
  // the ticket must start at zero (a normal call leaves it at zero; clear it anyway)
  cudaError_t e = cudaMemsetAsync(scratch + PARTIAL_BYTES, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return qxd::cuda_fail(nullptr, e, "cudaMemsetAsync(ticket)");
  const int grid = (int)((n + CHUNK - 1) / CHUNK);
  k_dot_noalloc<<<grid, THREADS, 0, st>>>((const double2*)a, (const double2*)b, (long long)n, scratch, out);
  e = cudaGetLastError();
  return e == cudaSuccess ? QXD_OK : qxd::cuda_fail(nullptr, e, "k_dot_noalloc launch");
}

// Forget the cached scratch addresses (host state only; no CUDA call).  After a device reset the
// library's module is loaded again and the array may move; the next qxd_vec_dot_noalloc then
// looks its address up afresh.
extern "C" qxd_status qxd_vec_dot_noalloc_forget(void) {
  std::lock_guard<std::mutex> lock(g_mutex);
  for (void*& a : g_scratch_addr) a = nullptr;
  return QXD_OK;
}
