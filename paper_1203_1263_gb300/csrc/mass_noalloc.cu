// nlse_mass_noalloc: the mass reduction for callers that cannot allocate
// device memory.
//
// Some callers are not allowed to call cudaMalloc at all: code that runs
// while another component is capturing the stream into a CUDA graph (an
// allocation there is illegal), plug-ins whose host application owns every
// byte of device memory through its own pool, and real-time loops that cannot
// afford the implicit device synchronisation an allocation may cause.  Such a
// caller cannot create a context (that needs a workspace buffer).  This entry
// point needs nothing but the input and one output double: its scratch (one
// pair of partial sums per block) lives in the file-scope array below, which
// every GPU that loads the library keeps until the process exits.
//
// The kernels are a variant of the context's mass reduction: each block sums a
// fixed run of sites with Neumaier's compensated summation, writes one
// (sum, compensation) pair into the scratch array, and a one-block second pass
// adds the pairs in a fixed order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdint.h>

#include <mutex>

#include "../../include/nlse.h"

namespace nlse {
void record_last_error(const char* msg);   // api.cu
}

namespace {

constexpr int kThreads = 256;
constexpr int kSitesPerBlock = 4096;     // each block sums this many sites
constexpr int kMaxBlocks = 8192;         // scratch capacity: 8192 pairs = 128 KiB
constexpr int kMaxDevices = 64;

// The scratch: one (sum, compensation) pair per block.  Every call writes each
// pair it later reads, so nothing needs clearing between calls; calls that
// overlap on the GPU (other streams, other host threads) race on it.
static __device__ __align__(256) double g_mass_scratch[2 * kMaxBlocks];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};   // device address of g_mass_scratch, per device

// Errors go to the library's nlse_last_error() buffer.
int fail(int code, const char* fmt, ...) {
  char msg[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  nlse::record_last_error(msg);
  return code;
}

struct Pair {
  double s, c;
};

__device__ __forceinline__ void nadd(Pair& a, double x) {
  const double t = a.s + x;
  if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x;
  else a.c += (x - t) + a.s;
  a.s = t;
}

__device__ __forceinline__ Pair block_sum(Pair v) {
  __shared__ double ss[kThreads / 32], sc[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double s = __shfl_down_sync(0xffffffffu, v.s, o), c = __shfl_down_sync(0xffffffffu, v.c, o);
    nadd(v, s);
    v.c += c;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { ss[warp] = v.s; sc[warp] = v.c; }
  __syncthreads();
  if (warp == 0) {
    v = (lane < kThreads / 32) ? Pair{ss[lane], sc[lane]} : Pair{0.0, 0.0};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double s = __shfl_down_sync(0xffffffffu, v.s, o), c = __shfl_down_sync(0xffffffffu, v.c, o);
      nadd(v, s);
      v.c += c;
    }
  }
  return v;
}

template <class C>
__global__ void __launch_bounds__(kThreads) k_mass_noalloc_blocks(const C* __restrict__ psi, int64_t total,
                                                                  double* scratch) {
  Pair acc = {0.0, 0.0};
  const int64_t base = (int64_t)blockIdx.x * kSitesPerBlock;
  for (int i = threadIdx.x; i < kSitesPerBlock; i += kThreads) {
    const int64_t p = base + i;
    if (p < total) {
      const C v = psi[p];
      const double x = double(v.x), y = double(v.y);
      nadd(acc, fma(x, x, y * y));
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = acc.s;
    scratch[2 * blockIdx.x + 1] = acc.c;
  }
}

__global__ void __launch_bounds__(kThreads) k_mass_noalloc_finish(const double* scratch, int nb, double scale,
                                                                  double* out) {
  Pair acc = {0.0, 0.0};
  for (int i = threadIdx.x; i < nb; i += kThreads) {
    nadd(acc, scratch[2 * i]);
    acc.c += scratch[2 * i + 1];
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[0] = scale * (acc.s + acc.c);
}

// Device address of the scratch array on the current device (set up once per
// device, on the first call made with that device current).
int scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(NLSE_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(NLSE_EINVAL, "device ordinal %d not supported", dev);
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mass_scratch);
    if (e != cudaSuccess || !p)
      return fail(NLSE_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return NLSE_OK;
}

}  // namespace

extern "C" {

int nlse_mass_noalloc(int dims, const int64_t* N, double h, int dtype, const void* psi, double* out, void* stream) {
  if (dims < 1 || dims > 3 || !N) return fail(NLSE_EINVAL, "dims must be 1..3 and N non-NULL");
  if (dtype != NLSE_C128 && dtype != NLSE_C64 && dtype != NLSE_C64_ACC64) return fail(NLSE_EINVAL, "bad dtype");
  if (!(h > 0) || !isfinite(h)) return fail(NLSE_EINVAL, "h must be > 0");
  if (!psi || !out) return fail(NLSE_EINVAL, "psi and out must be device pointers");
  // the site count, checked against the limit before each multiplication (no int64 overflow)
  const int64_t limit = (int64_t)kMaxBlocks * kSitesPerBlock;
  int64_t total = 1;
  for (int k = 0; k < dims; ++k)
    if (N[k] < 1) return fail(NLSE_EINVAL, "every N must be >= 1");
  for (int k = 0; k < dims; ++k) {
    if (N[k] > limit / total)
      return fail(NLSE_EINVAL, "grid exceeds the no-alloc maximum of %lld sites (%d blocks of %d sites)",
                  (long long)limit, kMaxBlocks, kSitesPerBlock);
    total *= N[k];
  }
  const int64_t nb = (total + kSitesPerBlock - 1) / kSitesPerBlock;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != NLSE_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == NLSE_C64)
    k_mass_noalloc_blocks<float2><<<(unsigned)nb, kThreads, 0, st>>>(static_cast<const float2*>(psi), total, scratch);
  else
    k_mass_noalloc_blocks<double2><<<(unsigned)nb, kThreads, 0, st>>>(static_cast<const double2*>(psi), total, scratch);
  k_mass_noalloc_finish<<<1, kThreads, 0, st>>>(scratch, (int)nb, pow(h, dims), out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(NLSE_ECUDA, "launch: %s", cudaGetErrorString(e));
  return NLSE_OK;
}

}  // extern "C"
