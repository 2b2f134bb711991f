// 1D grids of up to a few ten thousand sites: one thread-block cluster owns
// the whole line for every step of an nlse_step call.
//
// Such a line is a few hundred kilobytes at most, so every launch of the
// stage-streaming path is mostly latency (launch, dependency chain, a wave
// that fills a fraction of the GPU).  Here the CL CTAs of one cluster (CL up
// to 16, one per SM) each keep a contiguous segment of the line in shared
// memory: Psi^n, Psi_tmp, Psi_out (each with a two-site halo on either side)
// and K_tot.  A stage is a cluster barrier, a copy of the stage input's
// halo from the neighbouring CTAs' shared memory (distributed shared
// memory), a CTA barrier, and the segment's sites computed with the same
// per-site code (process_site, rk_apply) as every other kernel, so results
// are bit-for-bit those of the per-site kernel.  On the exact-sum stages the
// next step's fixed-point scale is derived, as elsewhere, from the largest
// exponent stage 4 wrote, here reduced across the cluster in rank 0's shared
// memory.  Psi is read from and written back to global memory once per call.
#pragma once
#include <cooperative_groups.h>

#include "nlse_device.cuh"

namespace nlse {

namespace cg = cooperative_groups;

constexpr int kLineMaxCluster = 16;

// A site's stencil operands in a CTA's segment array (element 0 = site seg0 - 2).
template <class T>
struct LineAcc {
  using R = typename T::R;
  using C = typename T::C;
  using C2 = typename V2<R>::t;
  const C* p;
  int o;   // the site's element
  int F;   // exact-sum stencil: this step's fraction bits
  __device__ __forceinline__ static C2 cv(const C v) { return {R(v.x), R(v.y)}; }
  __device__ __forceinline__ C2 at0() const { return cv(p[o]); }
  __device__ __forceinline__ C2 at1(int, int s) const { return cv(p[o + s]); }
  __device__ __forceinline__ C2 at2(int, int s, int, int t) const { return cv(p[o + s + t]); }
  __device__ __forceinline__ C2 atv(const int* v) const { return cv(p[o + v[0]]); }
  __device__ __forceinline__ longlong2 fx0() const { return fix2(make_double2(p[o].x, p[o].y), F); }
  __device__ __forceinline__ longlong2 fx1(int, int s) const { return fix2(make_double2(p[o + s].x, p[o + s].y), F); }
  __device__ __forceinline__ longlong2 fx2(int, int s, int, int t) const {
    return fix2(make_double2(p[o + s + t].x, p[o + s + t].y), F);
  }
  __device__ __forceinline__ int fixF() const { return F; }
};

template <class T>
struct LineArgs {
  StageArgs<T> A[4];   // stages 1..4 as the stage-streaming path builds them (Psi updated in place)
  int64_t nsteps;
  int n;               // sites of the line
  int seg;             // sites per CTA (the last CTA may have fewer, at least 2)
  int F0, fix_offset;  // exact-sum stages: reference fraction bits and the test offset (k_fix_update)
};

// Fraction bits for the largest biased exponent E of the state (as k_fix_update).
__device__ __forceinline__ int line_fix_from(unsigned int E, int Fprev, int F0, int offset) {
  if (E == 0u) return F0 + offset;
  if (E < 2047u) return 1075 - int(E) + offset;
  return Fprev;
}

template <class T, int ORDER, bool EXACT>
__global__ void __launch_bounds__(1024) k_line1d(const __grid_constant__ LineArgs<T> L) {
  using C = typename T::C;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char line_smem[];
  const int seg = L.seg, W = seg + 4;
  C* fpsi = reinterpret_cast<C*>(line_smem);   // Psi^n with halo
  C* ftmp = fpsi + W;                          // Psi_tmp with halo
  C* fout = ftmp + W;                          // Psi_out with halo
  C* kt = fout + W;                            // K_tot (no halo)
  unsigned int* emax = reinterpret_cast<unsigned int*>(kt + seg);   // [2]: stage 4's exponent, by step parity
  const int rank = int(cluster.block_rank()), ncta = int(cluster.num_blocks());
  const int seg0 = rank * seg, cnt = min(seg, L.n - seg0);
  const int last_cnt = L.n - (ncta - 1) * seg;
  const bool periodic = L.A[0].f.bc == BC_PERIODIC;
  const typename T::M* gpsi = L.A[0].master_in;   // the caller's Psi (global)

  for (int i = threadIdx.x; i < cnt; i += blockDim.x) fpsi[2 + i] = gpsi[seg0 + i];
  if (threadIdx.x < 2) emax[threadIdx.x] = 0u;
  int F = EXACT ? cur_fix(L.A[0].f) : 0;

  for (int64_t step = 0; step < L.nsteps; ++step) {
    const int par = int(step & 1);
    unsigned int ex = 0;
    for (int s = 0; s < 4; ++s) {
      C* X = s == 0 ? fpsi : (s == 2 ? fout : ftmp);   // the stage's stencil input
      cluster.sync();   // every CTA's writes of the previous stage are visible
      if (EXACT && s == 0 && step > 0) {   // the exponent the previous step's stage 4 left in rank 0
        const unsigned int* e0 = cluster.map_shared_rank(emax, 0);
        F = line_fix_from(e0[1 - par], F, L.F0, L.fix_offset);
        if (rank == 0 && threadIdx.x == 0) emax[par] = 0u;   // read by every CTA one step ago
      }
      if (threadIdx.x < 4) {   // two halo sites on either side, from the neighbouring segments
        const bool left = threadIdx.x < 2;
        const int q = threadIdx.x & 1;
        int nb = left ? rank - 1 : rank + 1;
        bool ok = nb >= 0 && nb < ncta;
        if (!ok && periodic) { nb = (nb + ncta) % ncta; ok = true; }
        if (ok) {
          const C* src = cluster.map_shared_rank(X, nb);
          const int nb_cnt = nb == ncta - 1 ? last_cnt : seg;
          // left halo: the neighbour's last two sites; right halo: its first two
          if (left) X[q] = src[2 + nb_cnt - 2 + q];
          else X[2 + cnt + q] = src[2 + q];
        }
      }
      __syncthreads();
      StageArgs<T> B = L.A[s];
      B.psin = fpsi + 2 - seg0;   // indexable by the global site index
      B.ktot = kt - seg0;
      B.out = (s == 0 || s == 2) ? ftmp + 2 - seg0 : (s == 1 ? fout + 2 - seg0 : nullptr);
      B.master = reinterpret_cast<typename T::M*>(fpsi + 2 - seg0);
      B.master_in = B.master;
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int c = seg0 + i;
        const int idx[1] = {c};
        LineAcc<T> acc;
        acc.p = X;
        acc.o = i + 2;
        acc.F = F;
        unsigned int e;
        if (periodic) e = process_site_periodic_acc<T, 1, ORDER, EXACT>(B, acc, idx, c);
        else if (c >= 1 && c <= L.n - 2) e = process_site<T, 1, ORDER, EXACT>(B, acc, idx, c);
        else e = 0u;   // boundary sites: served by their interior neighbour
        ex = max(ex, e);
      }
    }
    if (EXACT) {   // the largest exponent of Psi^{n+1} across the cluster, into rank 0's word for this step
      ex = __reduce_max_sync(0xffffffffu, ex);
      if ((threadIdx.x & 31) == 0 && ex) atomicMax(cluster.map_shared_rank(emax + par, 0), ex);
    }
  }
  cluster.sync();
  typename T::M* out = L.A[3].master;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) out[seg0 + i] = fpsi[2 + i];
  cluster.sync();   // no CTA leaves while others may still read its shared memory
}

}  // namespace nlse

namespace nlse {

// The cluster for an n-site line: CL CTAs (16 at most, about 32 sites each at least, so that a stage's
// per-site work is spread over as many SMs as the cluster allows) of seg sites, the last one with at
// least 2 (the halo a neighbour copies); false when a segment does not fit in shared memory (elem =
// bytes of one complex value).
inline bool line_plan(int n, size_t elem, int* cl, int* seg, size_t* smem) {
  int c = n / 32;
  c = c < 1 ? 1 : (c > kLineMaxCluster ? kLineMaxCluster : c);
  for (; c >= 1; --c) {
    const int s = (n + c - 1) / c;
    if (n - (c - 1) * s < 2) continue;
    const size_t b = (size_t)(3 * (s + 4) + s) * elem + 16;
    if (b > 200 * 1024) return false;
    *cl = c;
    *seg = s;
    *smem = b;
    return true;
  }
  return false;
}

template <class T, int ORDER, bool EXACT>
cudaError_t launch_line1d(const LineArgs<T>& L, int cl, size_t smem, cudaStream_t stream) {
  auto kern = k_line1d<T, ORDER, EXACT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && cl > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  int threads = (L.seg + 31) / 32 * 32;
  if (threads > 1024) threads = 1024;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cl, 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (clusters < 1) return cudaErrorInvalidConfiguration;   // cannot be co-scheduled: the caller falls back
  return cudaLaunchKernelEx(&cfg, kern, L);
}

}  // namespace nlse
