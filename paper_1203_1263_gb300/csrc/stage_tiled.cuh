// Tiled stage kernels: the same per-site arithmetic as the generic kernel
// (process_site), with the stencil operands read from shared memory.
//
// 3D: a CTA owns a TX x TY tile of (x, y) columns and marches along z over a
// chunk of planes.  Shared memory holds a ring of six planes, each the tile
// plus a 2-cell halo on every side; planes z-2 .. z+2 feed the stencil of
// plane z (the 2SHOC five-point form needs +-2 along every axis, the wall
// ghosts need the +-1 diagonals).  While plane z is computed, plane z+4 is
// already in flight into registers; it is stored into the slot of plane z-2
// after the compute, so one barrier per plane suffices.  Each element of Psi
// is read from global memory once per tile (plus the halo overlap).
//
// 2D: a CTA owns a TX x TY tile plus a 2-cell halo in shared memory.
//
// Both compute only the deep interior (every index in [2, N-3]); the wall
// shell is left to the shell kernel (stage_generic.cuh).
#pragma once
#include "nlse_device.cuh"

namespace nlse {

template <class T>
struct SAcc3 {
  using R = typename T::R;
  using C = typename T::C;
  using C2 = typename V2<R>::t;
  const C* p[5];   // planes z-2 .. z+2
  int w;           // row length of a plane (TX + 4)
  int o;           // offset of the thread's site inside a plane
  __device__ __forceinline__ static C2 cv(const C v) { return {R(v.x), R(v.y)}; }
  __device__ __forceinline__ int off(int k, int s) const { return k == 1 ? s * w : (k == 2 ? s : 0); }
  __device__ __forceinline__ C2 at0() const { return cv(p[2][o]); }
  __device__ __forceinline__ C2 at1(int k, int s) const {
    return k == 0 ? cv(p[2 + s][o]) : cv(p[2][o + off(k, s)]);
  }
  __device__ __forceinline__ C2 at2(int k, int s, int j, int t) const {
    const int dz = (k == 0 ? s : 0) + (j == 0 ? t : 0);
    return cv(p[2 + dz][o + off(k, s) + off(j, t)]);
  }
  __device__ __forceinline__ C2 atv(const int* v) const { return cv(p[2 + v[0]][o + v[1] * w + v[2]]); }
};

template <class T>
struct SAcc2 {
  using R = typename T::R;
  using C = typename T::C;
  using C2 = typename V2<R>::t;
  const C* p;
  int w, o;
  __device__ __forceinline__ static C2 cv(const C v) { return {R(v.x), R(v.y)}; }
  __device__ __forceinline__ int off(int k, int s) const { return k == 0 ? s * w : s; }
  __device__ __forceinline__ C2 at0() const { return cv(p[o]); }
  __device__ __forceinline__ C2 at1(int k, int s) const { return cv(p[o + off(k, s)]); }
  __device__ __forceinline__ C2 at2(int k, int s, int j, int t) const { return cv(p[o + off(k, s) + off(j, t)]); }
  __device__ __forceinline__ C2 atv(const int* v) const { return cv(p[o + v[0] * w + v[1]]); }
};

// Exact-sum variants: the shared tiles hold the fixed-point operands; FP64
// values (wall ghosts, MSD walls, out-of-range fallback) come from global.
template <class T, int D>
struct SAccX3 : GAcc<T, D> {
  const longlong2* p[5];
  int w, o;
  __device__ __forceinline__ SAccX3(const Field<T>& f_, int64_t c_) : GAcc<T, D>(f_, c_) {}
  __device__ __forceinline__ int off(int k, int s) const { return k == 1 ? s * w : (k == 2 ? s : 0); }
  __device__ __forceinline__ longlong2 fx0() const { return p[2][o]; }
  __device__ __forceinline__ longlong2 fx1(int k, int s) const { return k == 0 ? p[2 + s][o] : p[2][o + off(k, s)]; }
};

template <class T, int D>
struct SAccX2 : GAcc<T, D> {
  const longlong2* p;
  int w, o;
  __device__ __forceinline__ SAccX2(const Field<T>& f_, int64_t c_) : GAcc<T, D>(f_, c_) {}
  __device__ __forceinline__ longlong2 fx0() const { return p[o]; }
  __device__ __forceinline__ longlong2 fx1(int k, int s) const { return p[o + (k == 0 ? s * w : s)]; }
};

template <class T, bool EXACT> struct RingElem { using type = typename T::C; };
template <class T> struct RingElem<T, true> { using type = longlong2; };

template <bool EXACT, class C, class E>
__device__ __forceinline__ E ring_value(const C v, int F) {
  if constexpr (EXACT) return fix2(make_double2(v.x, v.y), F);
  else return v;
}

__device__ __forceinline__ int ring6(int z) { return ((z % 6) + 6) % 6; }

template <class T, int ORDER, int TX, int TY, bool EXACT>
__global__ void __launch_bounds__(TX* TY) k_stage3d_tiled(const StageArgs<T> A, int zc) {
  using C = typename T::C;
  using E = typename RingElem<T, EXACT>::type;
  constexpr int W = TX + 4, H = TY + 4, PS = W * H, NT = TX * TY, NPER = (PS + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E* ring = reinterpret_cast<E*>(smem_raw);
  const Field<T>& f = A.f;
  const int nz = f.n[0], ny = f.n[1], nx = f.n[2];
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int zb = 1 + blockIdx.z * zc;
  const int ze = min(zb + zc, nz - 1);   // planes [zb, ze) are computed
  const int64_t plane = (int64_t)ny * nx;
  const int F = EXACT ? cur_fix(f) : 0;
  unsigned int ex = 0;

  E regs[NPER];
  auto load = [&](int z) {
#pragma unroll
    for (int i = 0; i < NPER; ++i) {
      const int e = tid + i * NT;
      const int r = e / W, q = e - r * W;
      const int gy = y0 - 2 + r, gx = x0 - 2 + q;
      const bool ok = e < PS && z >= 0 && z < nz && gy >= 0 && gy < ny && gx >= 0 && gx < nx;
      regs[i] = ring_value<EXACT, C, E>(ok ? f.in[z * plane + (int64_t)gy * nx + gx] : C{0, 0}, F);
    }
  };
  auto store = [&](int z) {
    E* dst = ring + ring6(z) * PS;
#pragma unroll
    for (int i = 0; i < NPER; ++i) {
      const int e = tid + i * NT;
      if (e < PS) dst[e] = regs[i];
    }
  };

  for (int z = zb - 2; z <= zb + 2; ++z) {
    load(z);
    store(z);
  }
  load(zb + 3);
  __syncthreads();

  const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
  const bool deep_xy = gx >= 2 + A.xwall && gx <= nx - 3 - A.xwall && gy >= 2 && gy <= ny - 3;   // wall shell: shell kernel
  const int o = (threadIdx.y + 2) * W + threadIdx.x + 2;
  for (int z = zb; z < ze; ++z) {
    if (deep_xy && z >= 2 && z <= nz - 3) {
      const int idx[3] = {z, gy, gx};
      const int64_t c = z * plane + (int64_t)gy * nx + gx;
      if constexpr (EXACT) {
        SAccX3<T, 3> acc(f, c);
#pragma unroll
        for (int d = 0; d < 5; ++d) acc.p[d] = ring + ring6(z - 2 + d) * PS;
        acc.w = W;
        acc.o = o;
        const PointVals<T> pv = load_point<T, -1, true>(A, c, f.V != nullptr);
        const auto pc = acc.at0();
        const auto Nc = fma(f.sG, norm2(pc), -pv.v);   // units of cLF
        const auto aL = a_lap_exact_deep<T, 3, ORDER>(f, acc, idx, c, pc, Nc);
        ex = max(ex, rk_apply<T>(A, c, {-fma(Nc, pc.y, aL.y), fma(Nc, pc.x, aL.x)}, pv));
      } else {
        SAcc3<T> acc;
#pragma unroll
        for (int d = 0; d < 5; ++d) acc.p[d] = ring + ring6(z - 2 + d) * PS;
        acc.w = W;
        acc.o = o;
        const PointVals<T> pv = load_point<T>(A, c, f.V != nullptr);
        const auto pc = acc.at0();
        const auto Nc = fma(f.s, norm2(pc), -pv.v);
        const auto aL = a_lap_body<T, 3, ORDER, SAcc3<T>, false>(f, acc, idx, c, pc, Nc);
        rk_apply<T>(A, c, {-fma(Nc, pc.y, aL.y), fma(Nc, pc.x, aL.x)}, pv);
      }
    }
    if (z + 3 <= ze + 1) store(z + 3);   // the slot of plane z-3, last read one plane ago
    if (z + 4 <= ze + 1) load(z + 4);
    __syncthreads();
  }
  if (A.emax) emax_commit(A.emax, ex);
}

template <class T, int ORDER, int TX, int TY, bool EXACT>
__global__ void __launch_bounds__(TX* TY) k_stage2d_tiled(const StageArgs<T> A) {
  using C = typename T::C;
  using E = typename RingElem<T, EXACT>::type;
  constexpr int W = TX + 4, H = TY + 4, PS = W * H, NT = TX * TY, NPER = (PS + NT - 1) / NT;
  __shared__ __align__(16) E tile[PS];
  const Field<T>& f = A.f;
  const int ny = f.n[0], nx = f.n[1];
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
  const bool deep = gx >= 2 && gx <= nx - 3 && gy >= 2 && gy <= ny - 3;   // wall shell: shell kernel
  const int64_t c = (int64_t)gy * nx + gx;
  const int F = EXACT ? cur_fix(f) : 0;
  unsigned int ex = 0;
  PointVals<T> pv;   // requested before the tile, so that both latencies overlap
  if (deep) pv = load_point<T, -1, EXACT>(A, c, f.V != nullptr);
#pragma unroll
  for (int i = 0; i < NPER; ++i) {
    const int e = tid + i * NT;
    if (e < PS) {
      const int r = e / W, q = e - r * W;
      const int ty_ = y0 - 2 + r, tx_ = x0 - 2 + q;
      tile[e] = ring_value<EXACT, C, E>((ty_ >= 0 && ty_ < ny && tx_ >= 0 && tx_ < nx) ? f.in[(int64_t)ty_ * nx + tx_]
                                                                                       : C{0, 0}, F);
    }
  }
  __syncthreads();
  if (deep) {
    const int idx[2] = {gy, gx};
    if constexpr (EXACT) {
      SAccX2<T, 2> acc(f, c);
      acc.p = tile;
      acc.w = W;
      acc.o = (threadIdx.y + 2) * W + threadIdx.x + 2;
      const auto pc = acc.at0();
      const auto Nc = fma(f.sG, norm2(pc), -pv.v);   // units of cLF
      const auto aL = a_lap_exact_deep<T, 2, ORDER>(f, acc, idx, c, pc, Nc);
      ex = rk_apply<T>(A, c, {-fma(Nc, pc.y, aL.y), fma(Nc, pc.x, aL.x)}, pv);
    } else {
      SAcc2<T> acc;
      acc.p = tile;
      acc.w = W;
      acc.o = (threadIdx.y + 2) * W + threadIdx.x + 2;
      const auto pc = acc.at0();
      const auto Nc = fma(f.s, norm2(pc), -pv.v);
      const auto aL = a_lap_body<T, 2, ORDER, SAcc2<T>, false>(f, acc, idx, c, pc, Nc);
      rk_apply<T>(A, c, {-fma(Nc, pc.y, aL.y), fma(Nc, pc.x, aL.x)}, pv);
    }
  }
  if (A.emax) emax_commit(A.emax, ex);
}

// Tile shapes selectable at run time (tile_cfg); -1 picks the default.
struct Tile3Cfg { int tx, ty; };

template <class T, int ORDER, int TX, int TY, bool EXACT>
cudaError_t launch3d_tiled_shape(const StageArgs<T>& A, cudaStream_t stream) {
  const int nz = A.f.n[0], ny = A.f.n[1], nx = A.f.n[2];
  const int tiles = ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
  const int planes = nz - 2;
  int nzc = (152 * 8 + tiles - 1) / tiles;
  if (nzc > planes) nzc = planes;
  if (nzc < 1) nzc = 1;
  const int zc = (planes + nzc - 1) / nzc;
  nzc = (planes + zc - 1) / zc;
  const size_t smem = 6 * (TX + 4) * (TY + 4) * sizeof(typename RingElem<T, EXACT>::type);
  auto kern = k_stage3d_tiled<T, ORDER, TX, TY, EXACT>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, nzc);
  kern<<<grid, dim3(TX, TY), smem, stream>>>(A, zc);
  return cudaGetLastError();
}

template <class T, int ORDER, bool EXACT = false>
cudaError_t launch3d_tiled(const StageArgs<T>& A, int tile_cfg, cudaStream_t stream) {
  switch (tile_cfg) {
    case 1: return launch3d_tiled_shape<T, ORDER, 64, 4, EXACT>(A, stream);
    case 2: return launch3d_tiled_shape<T, ORDER, 32, 16, EXACT>(A, stream);
    case 3: return launch3d_tiled_shape<T, ORDER, 64, 8, EXACT>(A, stream);
    default: return launch3d_tiled_shape<T, ORDER, 32, 8, EXACT>(A, stream);
  }
}

template <class T, int ORDER, int TX, int TY, bool EXACT>
cudaError_t launch2d_tiled_shape(const StageArgs<T>& A, cudaStream_t stream) {
  const int ny = A.f.n[0], nx = A.f.n[1];
  dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, 1);
  k_stage2d_tiled<T, ORDER, TX, TY, EXACT><<<grid, dim3(TX, TY), 0, stream>>>(A);
  return cudaGetLastError();
}

template <class T, int ORDER, bool EXACT = false>
cudaError_t launch2d_tiled(const StageArgs<T>& A, int tile_cfg, cudaStream_t stream) {
  switch (tile_cfg) {
    case 1: return launch2d_tiled_shape<T, ORDER, 64, 4, EXACT>(A, stream);
    case 2: return launch2d_tiled_shape<T, ORDER, 32, 16, EXACT>(A, stream);
    case 3: return launch2d_tiled_shape<T, ORDER, 64, 8, EXACT>(A, stream);
    default: return launch2d_tiled_shape<T, ORDER, 32, 8, EXACT>(A, stream);
  }
}

}  // namespace nlse
