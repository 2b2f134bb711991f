// Generic stage kernel: one thread per interior site, all reads through the
// read-only cache.  Simple and dimension-agnostic; it is the correctness
// baseline that the tiled kernels are checked against, the kernel used for
// 1D grids, and the default for 3D grids too small to fill the GPU with the
// z-marching kernel's tiles (latency, not bandwidth, bounds those).
#pragma once
#include "nlse_device.cuh"

namespace nlse {

// I = index type of the site decode: uint32_t whenever the count fits
// (64-bit integer division is a long software sequence on the GPU).
template <class T, int D, int ORDER, bool EXACT, class I>
__global__ void __launch_bounds__(256) k_stage_generic(const StageArgs<T> A) {
  const int64_t t64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned int ex = 0;
  if (t64 < A.f.ninterior) {
    int idx[D];
    I rem = I(t64);
    int64_t c = 0;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
      const I mk = I(A.f.m[k]);
      const I q = rem % mk;
      rem /= mk;
      idx[k] = int(q) + 1;
      c += idx[k] * A.f.st[k];
    }
    const GAcc<T, D> acc(A.f, c);
    ex = process_site<T, D, ORDER, EXACT>(A, acc, idx, c);
  }
  if (A.emax) emax_commit(A.emax, ex);
}

// ---------------------------------------------------------------------------
// Wall shell: the interior sites within one cell of a wall (some index equal
// to 1 or N-2).  The tiled kernels compute only the deep interior (every
// index in [2, N-3]), where the stencil never reaches past a wall and no
// boundary site is served; the shell kernel computes the rest with the
// generic per-site code.  Sites are enumerated exactly, face by face: with
// interior extents a_k = N_k - 2, deep extents d_k = max(a_k - 2, 0) and
// c_k = a_k - d_k (2, or 1 when a_k == 1), the shell is
//   {i_0 in the c_0 outer layers} x a_1 x a_2
//   + d_0 x {i_1 in the c_1 outer layers} x a_2 + d_0 x d_1 x {c_2 outer layers}.
// ---------------------------------------------------------------------------
// P = periodic grid: every index is updated (first index 0, extent N), the
// shell is the two layers at each end of every axis (indices 0, 1, N-2, N-1,
// the sites whose +-2 neighbours wrap), and the deep region is [2, N-3] as in
// the bounded case.
template <class T, int D, class I, bool P = false>
__device__ __forceinline__ int64_t shell_decode(const Field<T>& f, I t, int* idx) {
  constexpr int CF = P ? 4 : 2, LO = P ? 0 : 1;   // shell layers per axis (full), first updated index
  int a[3], d[3], c[3];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    a[k] = P ? f.n[k] : f.m[k];
    d[k] = a[k] > CF ? a[k] - CF : 0;
    c[k] = a[k] - d[k];
  }
  // q-th outer layer of axis k: the first CF/2 and the last CF/2 updated indices (all of them when d == 0)
  auto outer = [&](int k, int q) { return d[k] == 0 ? LO + q : (q < CF / 2 ? LO + q : LO + a[k] - CF + q); };
  if constexpr (D == 1) {
    idx[0] = outer(0, int(t));
  } else if constexpr (D == 2) {
    const I F0 = I(c[0]) * I(a[1]);
    if (t < F0) {
      idx[0] = outer(0, int(t / I(a[1])));
      idx[1] = LO + int(t % I(a[1]));
    } else {
      t -= F0;
      idx[0] = 2 + int(t / I(c[1]));
      idx[1] = outer(1, int(t % I(c[1])));
    }
  } else {
    const I F0 = I(c[0]) * I(a[1]) * I(a[2]);
    const I F1 = I(d[0]) * I(c[1]) * I(a[2]);
    if (t < F0) {
      const I pa = I(a[1]) * I(a[2]);
      idx[0] = outer(0, int(t / pa));
      const I r = t % pa;
      idx[1] = LO + int(r / I(a[2]));
      idx[2] = LO + int(r % I(a[2]));
    } else if (t < F0 + F1) {
      t -= F0;
      const I pa = I(c[1]) * I(a[2]);
      idx[0] = 2 + int(t / pa);
      const I r = t % pa;
      idx[1] = outer(1, int(r / I(a[2])));
      idx[2] = LO + int(r % I(a[2]));
    } else {
      t -= F0 + F1;
      const I pa = I(d[1]) * I(c[2]);
      idx[0] = 2 + int(t / pa);
      const I r = t % pa;
      idx[1] = 2 + int(r / I(c[2]));
      idx[2] = outer(2, int(r % I(c[2])));
    }
  }
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) s += idx[k] * f.st[k];
  return s;
}

// Sites of the shell: a = updated extents (N - 2, or N on a periodic grid), cf = shell layers per axis.
inline int64_t shell_count(int D, const int* a, int cf = 2) {
  int64_t all = 1, deep = 1;
  for (int k = 0; k < D; ++k) {
    all *= a[k];
    deep *= (a[k] > cf ? a[k] - cf : 0);
  }
  return all - deep;
}

inline bool has_deep(int D, const int* m) {
  for (int k = 0; k < D; ++k)
    if (m[k] <= 2) return false;
  return true;
}

template <class T, int D, int ORDER, bool EXACT, class I>
__global__ void __launch_bounds__(256) k_stage_shell(const StageArgs<T> A, int64_t nshell) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned int ex = 0;
  if (t < nshell) {
    int idx[D];
    const int64_t c = shell_decode<T, D, I>(A.f, I(t), idx);
    const GAcc<T, D> acc(A.f, c);
    ex = process_site<T, D, ORDER, EXACT>(A, acc, idx, c);
  }
  if (A.emax) emax_commit(A.emax, ex);
}

// CTA size of the one-thread-per-site kernels: 256 threads, halved (down to
// one warp) while the grid would give fewer than two CTAs per SM.  On small
// grids this spreads the sites over all SMs, which matters most on the FP64
// path (a few FP64 instructions per cycle per SM); it never changes results.
inline int site_kernel_threads(int64_t n) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      sms = v;
    else
      sms = 152;
  }
  int t = 256;
  while (t > 32 && (n + t - 1) / t < 2 * (int64_t)sms) t >>= 1;
  return t;
}

// Periodic grids: the shell (P) or every site (generic); each site's own multi-index, wrapped neighbours.
template <class T, int D, int ORDER, bool EXACT, class I>
__global__ void __launch_bounds__(256) k_stage_shell_periodic(const StageArgs<T> A, int64_t nshell) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned int ex = 0;
  if (t < nshell) {
    int idx[D];
    const int64_t c = shell_decode<T, D, I, true>(A.f, I(t), idx);
    ex = process_site_periodic<T, D, ORDER, EXACT>(A, idx, c);
  }
  if (A.emax) emax_commit(A.emax, ex);
}

template <class T, int D, int ORDER, bool EXACT, class I>
__global__ void __launch_bounds__(256) k_stage_generic_periodic(const StageArgs<T> A, int64_t total) {
  const int64_t t64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned int ex = 0;
  if (t64 < total) {
    int idx[D];
    I rem = I(t64);
    int64_t c = 0;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
      const I nk = I(A.f.n[k]);
      idx[k] = int(rem % nk);
      rem /= nk;
      c += idx[k] * A.f.st[k];
    }
    ex = process_site_periodic<T, D, ORDER, EXACT>(A, idx, c);
  }
  if (A.emax) emax_commit(A.emax, ex);
}

template <class T, int D, int ORDER, bool EXACT = false>
cudaError_t launch_shell(const StageArgs<T>& A, cudaStream_t stream) {
  const int64_t ns = shell_count(D, A.f.m);
  if (ns <= 0) return cudaSuccess;
  const int threads = site_kernel_threads(ns);
  const dim3 grid((unsigned)((ns + threads - 1) / threads));
  if (A.f.ninterior < (int64_t(1) << 31)) k_stage_shell<T, D, ORDER, EXACT, uint32_t><<<grid, threads, 0, stream>>>(A, ns);
  else k_stage_shell<T, D, ORDER, EXACT, uint64_t><<<grid, threads, 0, stream>>>(A, ns);
  return cudaGetLastError();
}

template <class T, int D, int ORDER, bool EXACT = false>
cudaError_t launch_shell_periodic(const StageArgs<T>& A, cudaStream_t stream) {
  const int64_t ns = shell_count(D, A.f.n, 4);
  if (ns <= 0) return cudaSuccess;
  const int threads = site_kernel_threads(ns);
  const dim3 grid((unsigned)((ns + threads - 1) / threads));
  if (ns < (int64_t(1) << 31)) k_stage_shell_periodic<T, D, ORDER, EXACT, uint32_t><<<grid, threads, 0, stream>>>(A, ns);
  else k_stage_shell_periodic<T, D, ORDER, EXACT, uint64_t><<<grid, threads, 0, stream>>>(A, ns);
  return cudaGetLastError();
}

template <class T, int D, int ORDER, bool EXACT = false>
cudaError_t launch_generic_periodic(const StageArgs<T>& A, cudaStream_t stream) {
  int64_t total = 1;
  for (int k = 0; k < D; ++k) total *= A.f.n[k];
  const int threads = site_kernel_threads(total);
  const int64_t blocks = (total + threads - 1) / threads;
  if (total < (int64_t(1) << 31))
    k_stage_generic_periodic<T, D, ORDER, EXACT, uint32_t><<<dim3((unsigned)blocks), threads, 0, stream>>>(A, total);
  else
    k_stage_generic_periodic<T, D, ORDER, EXACT, uint64_t><<<dim3((unsigned)blocks), threads, 0, stream>>>(A, total);
  return cudaGetLastError();
}

template <class T, int D, int ORDER, bool EXACT = false>
cudaError_t launch_generic(const StageArgs<T>& A, cudaStream_t stream) {
  if (A.f.ninterior <= 0) return cudaSuccess;
  const int threads = site_kernel_threads(A.f.ninterior);
  const int64_t blocks = (A.f.ninterior + threads - 1) / threads;
  if (A.f.ninterior < (int64_t(1) << 31))
    k_stage_generic<T, D, ORDER, EXACT, uint32_t><<<dim3((unsigned)blocks), threads, 0, stream>>>(A);
  else
    k_stage_generic<T, D, ORDER, EXACT, uint64_t><<<dim3((unsigned)blocks), threads, 0, stream>>>(A);
  return cudaGetLastError();
}

}  // namespace nlse
