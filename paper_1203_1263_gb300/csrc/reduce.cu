// FP64 reductions: mass, energy and max|V|.
//
// Each thread accumulates with Neumaier's compensated summation (Neumaier
// 1974), pairs (sum, compensation) are combined by warp shuffles and through
// shared memory, every block writes one pair, and a single-block second pass
// adds the block pairs in a fixed order, so a result depends only on the
// input, never on scheduling.
#include "nlse_device.cuh"
#include "nlse_internal.h"

namespace nlse {

struct Neu {
  double s, c;
};

__device__ __forceinline__ void nadd(Neu& a, double x) {
  const double t = a.s + x;
  if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x;
  else a.c += (x - t) + a.s;
  a.s = t;
}

__device__ __forceinline__ void nmerge(Neu& a, const Neu& b) {
  nadd(a, b.s);
  a.c += b.c;
}

// Block-wide combination; thread 0 gets the block's pair.
__device__ __forceinline__ Neu block_reduce(Neu v) {
  __shared__ double ss[32], sc[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Neu w = {__shfl_down_sync(0xffffffffu, v.s, o), __shfl_down_sync(0xffffffffu, v.c, o)};
    nmerge(v, w);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) { ss[warp] = v.s; sc[warp] = v.c; }
  __syncthreads();
  if (warp == 0) {
    v = (lane < nw) ? Neu{ss[lane], sc[lane]} : Neu{0.0, 0.0};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Neu w = {__shfl_down_sync(0xffffffffu, v.s, o), __shfl_down_sync(0xffffffffu, v.c, o)};
      nmerge(v, w);
    }
  }
  return v;
}

template <class C>
__global__ void __launch_bounds__(256) k_mass(const C* __restrict__ psi, int64_t total, double* partials,
                                              unsigned int* flag) {
  Neu acc = {0.0, 0.0};
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 p = ld2<double>(psi, i);
    const double m2 = norm2(p);
    bad |= !isfinite(m2);
    nadd(acc, m2);
  }
  if (bad) atomicOr(flag, 2u);
  acc = block_reduce(acc);
  if (threadIdx.x == 0) { partials[2 * blockIdx.x] = acc.s; partials[2 * blockIdx.x + 1] = acc.c; }
}

template <class T, int D, int ORDER>
__global__ void __launch_bounds__(256) k_energy(const Field<T> f, double* partials, unsigned int* flag) {
  Neu acc = {0.0, 0.0};
  bool bad = false;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < f.ninterior;
       t += (int64_t)gridDim.x * blockDim.x) {
    int idx[D];
    int64_t rem = t, c = 0;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
      const int64_t q = rem % f.m[k];
      rem /= f.m[k];
      idx[k] = int(q) + 1;
      c += idx[k] * f.st[k];
    }
    const double2 pc = ld2<double>(f.in, c);
    const double m2 = norm2(pc);
    const double v = ldv<double>(f.V, c);
    const double Nc = fma(f.s, m2, -v);
    const GAcc<T, D> ga(f, c);
    const double2 aL = a_lap<T, D, ORDER>(f, ga, idx, c, pc, Nc);
    const double e = fma(-0.5 * f.s, m2 * m2, fma(v, m2, -fma(pc.x, aL.x, pc.y * aL.y)));
    bad |= !isfinite(e);
    nadd(acc, e);
  }
  if (bad) atomicOr(flag, 2u);
  acc = block_reduce(acc);
  if (threadIdx.x == 0) { partials[2 * blockIdx.x] = acc.s; partials[2 * blockIdx.x + 1] = acc.c; }
}

// Periodic grids: every site counts, neighbours wrap.
template <class T, int D, int ORDER>
__global__ void __launch_bounds__(256) k_energy_periodic(const Field<T> f, int64_t total, double* partials,
                                                         unsigned int* flag) {
  Neu acc = {0.0, 0.0};
  bool bad = false;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int idx[D];
    int64_t rem = t, c = 0;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
      idx[k] = int(rem % f.n[k]);
      rem /= f.n[k];
      c += idx[k] * f.st[k];
    }
    const double2 pc = ld2<double>(f.in, c);
    const double m2 = norm2(pc);
    const double v = ldv<double>(f.V, c);
    const double Nc = fma(f.s, m2, -v);
    const GAccP<T, D> ga(f, c, idx);
    const double2 aL = a_lap_body<T, D, ORDER, GAccP<T, D>, false>(f, ga, idx, c, pc, Nc);
    const double e = fma(-0.5 * f.s, m2 * m2, fma(v, m2, -fma(pc.x, aL.x, pc.y * aL.y)));
    bad |= !isfinite(e);
    nadd(acc, e);
  }
  if (bad) atomicOr(flag, 2u);
  acc = block_reduce(acc);
  if (threadIdx.x == 0) { partials[2 * blockIdx.x] = acc.s; partials[2 * blockIdx.x + 1] = acc.c; }
}

// Second pass: one block adds the nb block pairs in a fixed order.
__global__ void __launch_bounds__(256) k_finish(const double* partials, int nb, double scale, double* result) {
  Neu acc = {0.0, 0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) nmerge(acc, Neu{partials[2 * i], partials[2 * i + 1]});
  acc = block_reduce(acc);
  if (threadIdx.x == 0) result[0] = scale * (acc.s + acc.c);
}

template <class VR>
__global__ void __launch_bounds__(256) k_vmax(const VR* __restrict__ V, int64_t total, unsigned long long* out) {
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(double(V[i])));
  // non-negative doubles order like their bit patterns
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// Largest biased exponent over the components of a complex128 array into *out
// (exact-sum scale of the current state; *out must start at 0).
__global__ void __launch_bounds__(256) k_max_expo(const double* __restrict__ v, int64_t n, unsigned int* out) {
  unsigned int e = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    e = max(e, expo_bits(__ldg(v + i)));
  emax_commit(out, e);
}

// Fraction bits of the exact-sum stencil for the state whose largest
// component has biased exponent E (collected in *emax by k_max_expo or by
// stage 4): |v| < 2^(E - 1022), so F = 1075 - E keeps every component below
// 2^53 in fixed point, 4x below the accepted range 2^55.  A zero state keeps F0;
// a non-finite one keeps the previous F (the non-finite flag reports it).
// `offset` is a test hook (nlse_debug_set).  Resets *emax for the next step.
__global__ void k_fix_update(unsigned int* emax, int* fdev, int F0, int offset) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const unsigned int E = *emax;
    if (E == 0u) *fdev = F0 + offset;
    else if (E < 2047u) *fdev = 1075 - int(E) + offset;
    *emax = 0u;
  }
}

cudaError_t launch_fix_update(const double* psi, int64_t n, unsigned int* emax, int* fdev, int F0, int offset,
                              cudaStream_t stream) {
  if (psi) {
    int64_t b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    k_max_expo<<<(unsigned)b, 256, 0, stream>>>(psi, n, emax);
  }
  k_fix_update<<<1, 32, 0, stream>>>(emax, fdev, F0, offset);
  return cudaGetLastError();
}

static int reduce_blocks(int64_t work) {
  int64_t b = (work + 256 * 8 - 1) / (256 * 8);
  if (b < 1) b = 1;
  if (b > kMaxReduceBlocks) b = kMaxReduceBlocks;
  return int(b);
}

cudaError_t launch_mass(const void* psi, bool psi_double, int64_t total, double scale, double* partials,
                        double* result, unsigned int* flag, cudaStream_t stream) {
  const int nb = reduce_blocks(total);
  if (psi_double) k_mass<double2><<<nb, 256, 0, stream>>>((const double2*)psi, total, partials, flag);
  else k_mass<float2><<<nb, 256, 0, stream>>>((const float2*)psi, total, partials, flag);
  k_finish<<<1, 256, 0, stream>>>(partials, nb, scale, result);
  return cudaGetLastError();
}

template <class T, int D, int ORDER>
cudaError_t launch_energy(const Field<T>& f, double scale, double* partials, double* result, unsigned int* flag,
                          cudaStream_t stream) {
  if (f.bc == BC_PERIODIC) {
    int64_t total = 1;
    for (int k = 0; k < D; ++k) total *= f.n[k];
    const int nb = reduce_blocks(total);
    k_energy_periodic<T, D, ORDER><<<nb, 256, 0, stream>>>(f, total, partials, flag);
    k_finish<<<1, 256, 0, stream>>>(partials, nb, scale, result);
    return cudaGetLastError();
  }
  const int nb = reduce_blocks(f.ninterior);
  k_energy<T, D, ORDER><<<nb, 256, 0, stream>>>(f, partials, flag);
  k_finish<<<1, 256, 0, stream>>>(partials, nb, scale, result);
  return cudaGetLastError();
}

#define INST(T, D, O) \
  template cudaError_t launch_energy<T, D, O>(const Field<T>&, double, double*, double*, unsigned int*, cudaStream_t);
INST(P64, 1, 2) INST(P64, 1, 4) INST(P64, 2, 2) INST(P64, 2, 4) INST(P64, 3, 2) INST(P64, 3, 4)
INST(E32, 1, 2) INST(E32, 1, 4) INST(E32, 2, 2) INST(E32, 2, 4) INST(E32, 3, 2) INST(E32, 3, 4)
INST(EMix, 1, 2) INST(EMix, 1, 4) INST(EMix, 2, 2) INST(EMix, 2, 4) INST(EMix, 3, 2) INST(EMix, 3, 4)
#undef INST

cudaError_t launch_vmax(const void* V, bool v_double, int64_t total, unsigned long long* out, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  const int nb = reduce_blocks(total);
  if (v_double) k_vmax<double><<<nb, 256, 0, stream>>>((const double*)V, total, out);
  else k_vmax<float><<<nb, 256, 0, stream>>>((const float*)V, total, out);
  return cudaGetLastError();
}

}  // namespace nlse
