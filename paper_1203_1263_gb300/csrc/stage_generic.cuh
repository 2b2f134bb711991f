// Generic stage kernel: one thread per interior site, all reads through the
// read-only cache.  Simple and dimension-agnostic; it is the correctness
// baseline that the tiled kernels are checked against, and the kernel used
// for 1D grids.
#pragma once
#include "nlse_device.cuh"

namespace nlse {

template <class T, int D, int ORDER>
__global__ void __launch_bounds__(256) k_stage_generic(const StageArgs<T> A) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.f.ninterior) return;
  int idx[D];
  int64_t rem = t, c = 0;
#pragma unroll
  for (int k = D - 1; k >= 0; --k) {
    const int64_t q = rem % A.f.m[k];
    rem /= A.f.m[k];
    idx[k] = int(q) + 1;
    c += idx[k] * A.f.st[k];
  }
  const GAcc<T, D> acc(A.f, c);
  process_site<T, D, ORDER>(A, acc, idx, c);
}

template <class T, int D, int ORDER>
cudaError_t launch_generic(const StageArgs<T>& A, cudaStream_t stream) {
  if (A.f.ninterior <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (A.f.ninterior + threads - 1) / threads;
  k_stage_generic<T, D, ORDER><<<dim3((unsigned)blocks), threads, 0, stream>>>(A);
  return cudaGetLastError();
}

}  // namespace nlse
