// Wall-shell sites of a 3D grid, processed as thin slabs along each wall
// with the stage input staged in shared memory.
//
// The shell takes the interior sites within one cell of the z and y walls and
// within three cells of the x walls ("marching" names a slab's long axis):
//   z-walls  z in {1, Nz-2},  y in [1, Ny-2], x in [1, Nx-2]          marching y, normal z, fast x
//   y-walls  z in [2, Nz-3],  y in {1, Ny-2}, x in [1, Nx-2]          marching z, normal y, fast x
//   x-walls  z in [2, Nz-3],  y in [2, Ny-3], x in {1,2,3, Nx-4..Nx-2} marching z, normal x, fast y
// and the deep-interior kernels then start at x = 4 (StageArgs::xwall = 2).
// The wider x-wall slab owns every site of the 32-byte rows x = 0..3 (and
// their mirror), so the pointwise arrays of those rows are fetched by one
// kernel only.
// (The FP64 path keeps one x layer: there the deep kernel's exact-sum stencil
// is cheaper per site than the slab's, and the FP64 pipe, not DRAM, bounds it.)
// A CTA owns TF consecutive fast coordinates of one wall and MC consecutive
// marching coordinates, one thread per site.  Its window holds, for each of
// the MC + 4 marching planes m0-2 .. m0+MC+1, the NS + 3 layers next to the
// wall by TF + 4 fast coordinates (two of halo each side), zero outside the
// grid, staged in shared memory once.  The per-site arithmetic is the same
// process_site code as every other kernel, through an accessor over the
// window, so results are bit-identical to the global-memory shell kernel.
// Requires extents >= 7 (z, y) and >= 10 (x).
#pragma once
#include "nlse_device.cuh"

namespace nlse {

template <class T, int AXM, int AXN, int AXF>
struct SlabAcc {
  using R = typename T::R;
  using C = typename T::C;
  using C2 = typename V2<R>::t;
  const C* p[5];   // planes m-2 .. m+2
  int wf;          // fast extent of a plane (TF + 4)
  int o;           // the site's index inside a plane
  int F;           // fixed-point fraction bits (exact-sum stencil)
  __device__ __forceinline__ static C2 cv(const C v) { return {R(v.x), R(v.y)}; }
  __device__ __forceinline__ int off(int k, int s) const { return k == AXN ? s * wf : (k == AXF ? s : 0); }
  __device__ __forceinline__ C2 at0() const { return cv(p[2][o]); }
  __device__ __forceinline__ C2 at1(int k, int s) const {
    return k == AXM ? cv(p[2 + s][o]) : cv(p[2][o + off(k, s)]);
  }
  __device__ __forceinline__ C2 at2(int k, int s, int j, int t) const {
    const int dm = (k == AXM ? s : 0) + (j == AXM ? t : 0);
    return cv(p[2 + dm][o + off(k, s) + off(j, t)]);
  }
  __device__ __forceinline__ C2 atv(const int* v) const { return cv(p[2 + v[AXM]][o + v[AXN] * wf + v[AXF]]); }
  __device__ __forceinline__ longlong2 fx0() const { return fix2(make_double2(p[2][o].x, p[2][o].y), F); }
  __device__ __forceinline__ longlong2 fx1(int k, int s) const {
    const C v = k == AXM ? p[2 + s][o] : p[2][o + off(k, s)];
    return fix2(make_double2(v.x, v.y), F);
  }
  __device__ __forceinline__ longlong2 fx2(int k, int s, int j, int t) const {
    const C2 v = at2(k, s, j, t);
    return fix2(make_double2(v.x, v.y), F);
  }
  __device__ __forceinline__ int fixF() const { return F; }
};

struct SlabRange {
  int m_lo, m_hi;   // site range along the marching axis (inclusive)
  int f_lo, f_hi;   // site range along the fast axis (inclusive)
};

constexpr int kSlabTF = 32;
template <int NS> struct SlabShape {
  static constexpr int MC = NS == 1 ? 8 : 4;     // marching sites per CTA
  static constexpr int NWL = NS + 3;             // window layers along the normal axis
  static constexpr int THREADS = NS * kSlabTF * MC;
};

// blockIdx.x: fast tile, blockIdx.y: marching block, blockIdx.z: 0 = low wall, 1 = high wall.
// NS sites per (marching, fast) position along the normal axis: low wall 1 .. NS,
// high wall N-1-NS .. N-2.  Thread (tn, tf, tm), tn fastest, processes site
// (m0 + tm, normal site tn, f0 + tf).
// S: the RK4 stage (compile time, so that only that stage's update is in the kernel's code).
template <class T, int ORDER, bool EXACT, int AXM, int AXN, int AXF, int NS, int S>
__global__ void __launch_bounds__(SlabShape<NS>::THREADS) k_stage_slab(const StageArgs<T> A, const SlabRange rg) {
  using C = typename T::C;
  using Sh = SlabShape<NS>;
  constexpr int WF = kSlabTF + 4, NWL = Sh::NWL, PL = NWL * WF, NP = Sh::MC + 4;
  __shared__ C win[NP * PL];
  const Field<T>& f = A.f;
  const int tid = threadIdx.x;
  const bool hi = blockIdx.z != 0;
  const int n_win0 = hi ? f.n[AXN] - NWL : 0;        // first of the window's normal layers
  const int n_first = hi ? f.n[AXN] - 1 - NS : 1;    // first site layer
  const int f0 = rg.f_lo + blockIdx.x * kSlabTF;     // first site of this CTA along the fast axis
  const int m0 = rg.m_lo + blockIdx.y * Sh::MC;       // first site along the marching axis

  for (int e = tid; e < NP * PL; e += Sh::THREADS) {
    const int pl = e / PL, r = e % PL;
    int nw, fw;
    if (AXF == 2) { nw = r / WF; fw = r % WF; }       // fast axis contiguous in memory
    else { fw = r / NWL; nw = r % NWL; }              // normal axis contiguous (x walls)
    const int m = m0 - 2 + pl, fc = f0 - 2 + fw;
    C v;
    v.x = 0;
    v.y = 0;
    if (m >= 0 && m < f.n[AXM] && fc >= 0 && fc < f.n[AXF])
      v = f.in[(int64_t)m * f.st[AXM] + (int64_t)(n_win0 + nw) * f.st[AXN] + (int64_t)fc * f.st[AXF]];
    win[pl * PL + nw * WF + fw] = v;
  }
  __syncthreads();
  // tn fastest: the x-wall layers of one row are adjacent lanes (their pointwise
  // operands share 32-byte sectors)
  const int tn = tid % NS, tf = (tid / NS) % kSlabTF, tm = tid / (NS * kSlabTF);
  const int fs = f0 + tf, ms = m0 + tm, ns = n_first + tn;
  unsigned int ex = 0;
  if (fs <= rg.f_hi && ms <= rg.m_hi) {
    int idx[3];
    idx[AXM] = ms;
    idx[AXN] = ns;
    idx[AXF] = fs;
    const int64_t c = (int64_t)idx[0] * f.st[0] + (int64_t)idx[1] * f.st[1] + (int64_t)idx[2] * f.st[2];
    SlabAcc<T, AXM, AXN, AXF> acc;
#pragma unroll
    for (int k = 0; k < 5; ++k) acc.p[k] = win + (tm + k) * PL;
    acc.wf = WF;
    acc.o = (ns - n_win0) * WF + (tf + 2);
    acc.F = EXACT ? cur_fix(f) : 0;
    ex = process_site<T, 3, ORDER, EXACT, SlabAcc<T, AXM, AXN, AXF>, S>(A, acc, idx, c);
  }
  if (A.emax) emax_commit(A.emax, ex);
}

inline bool slab_ok(const int* n) { return n[0] >= 7 && n[1] >= 7 && n[2] >= 10; }

template <class T, int ORDER, bool EXACT, int AXM, int AXN, int AXF, int NS>
cudaError_t launch_slab(const StageArgs<T>& A, const SlabRange& rg, cudaStream_t stream) {
  using Sh = SlabShape<NS>;
  const dim3 grid((unsigned)((rg.f_hi - rg.f_lo) / kSlabTF + 1), (unsigned)((rg.m_hi - rg.m_lo) / Sh::MC + 1), 2);
  switch (A.stage) {
    case 1: k_stage_slab<T, ORDER, EXACT, AXM, AXN, AXF, NS, 1><<<grid, Sh::THREADS, 0, stream>>>(A, rg); break;
    case 2: k_stage_slab<T, ORDER, EXACT, AXM, AXN, AXF, NS, 2><<<grid, Sh::THREADS, 0, stream>>>(A, rg); break;
    case 3: k_stage_slab<T, ORDER, EXACT, AXM, AXN, AXF, NS, 3><<<grid, Sh::THREADS, 0, stream>>>(A, rg); break;
    case 4: k_stage_slab<T, ORDER, EXACT, AXM, AXN, AXF, NS, 4><<<grid, Sh::THREADS, 0, stream>>>(A, rg); break;
    default: k_stage_slab<T, ORDER, EXACT, AXM, AXN, AXF, NS, -1><<<grid, Sh::THREADS, 0, stream>>>(A, rg); break;
  }
  return cudaGetLastError();
}

// The whole 3D shell as three slab launches (axes: 0 = z, 1 = y, 2 = x); with
// NSX = 3 x-wall layers the caller's deep-interior kernels must run with
// xwall = 2, with NSX = 1 with xwall = 0.
// yx: if given, the y- and x-wall slabs go to yx[0] and yx[1] (all three slabs then run concurrently).
template <class T, int ORDER, bool EXACT, int NSX>
cudaError_t launch_shell_slabs(const StageArgs<T>& A, cudaStream_t stream, const cudaStream_t* yx = nullptr) {
  const int* n = A.f.n;
  cudaError_t e;
  // z walls: march y over [1, Ny-2], fast x over [1, Nx-2]
  if ((e = launch_slab<T, ORDER, EXACT, 1, 0, 2, 1>(A, SlabRange{1, n[1] - 2, 1, n[2] - 2}, stream)) != cudaSuccess)
    return e;
  // y walls: march z over [2, Nz-3], fast x over [1, Nx-2]
  if ((e = launch_slab<T, ORDER, EXACT, 0, 1, 2, 1>(A, SlabRange{2, n[0] - 3, 1, n[2] - 2},
                                                    yx && yx[0] ? yx[0] : stream)) != cudaSuccess)
    return e;
  // x walls (NSX layers each): march z over [2, Nz-3], fast y over [2, Ny-3]
  return launch_slab<T, ORDER, EXACT, 0, 2, 1, NSX>(A, SlabRange{2, n[0] - 3, 2, n[1] - 3},
                                                    yx && yx[1] ? yx[1] : stream);
}

}  // namespace nlse
