// 3D z-marching stage kernel fed by the Tensor Memory Accelerator.
//
// A CTA owns a TX x TY tile of (x, y) columns and marches along z.  Each
// plane of the stage input, with a 2-cell halo on every side, arrives in
// shared memory by one cp.async.bulk.tensor load (out-of-range parts are
// zero-filled by the hardware, so there is no per-element bounds logic).  A
// ring of 5 + P slots keeps planes z-2 .. z+2 for the stencil while planes up
// to z+2+P are already in flight, each slot with its own mbarrier that the
// copy completes with its byte count; slots are used round-robin, so slot
// pointers and barrier phases advance without any index arithmetic.  The
// pointwise operands of the next plane (V, Psi^n, K_tot, master) are loaded
// into registers one plane ahead.  Each thread computes RY rows of the tile.
// Only deep-interior sites (two or more cells from every wall) are computed
// here, with no wall logic at all; the wall shell is the shell kernel's (the
// same arithmetic functions as every other kernel, so results are
// bit-identical).
// The stage is a template parameter.  One __syncthreads per plane releases
// the slot of plane z-2 for the load of plane z-2+RS.  Every wait on an mbarrier is bounded: if a copy never lands,
// the CTA records kFlagTimeout, waits (bounded) for its copies in flight and
// exits.
#pragma once
#include <cuda.h>

#include "nlse_device.cuh"
#include "nlse_internal.h"
#include "stage_tiled.cuh"

namespace nlse {

constexpr unsigned int kFlagTimeout = 4u;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the barrier; false after `limit` cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

template <int TX, int TY, class C>
struct TmaGeom {
  static constexpr int W = TX + 4, H = TY + 4, PS = W * H;
  static constexpr uint32_t kBytes = PS * sizeof(C);                       // one plane with halo
  static constexpr uint32_t kSlot = (kBytes + 127u) / 128u * 128u;         // 128-byte aligned slots
};

// Number of z chunks for a z-marching kernel over `tiles` (x, y) tiles and
// `planes` planes, `per_sm` CTAs resident per SM: the count whose waves times
// planes per CTA (plus the `fill` planes a chunk's ring loads before its
// first output plane) is least, so that no short last wave or overlong
// chunk sets the kernel's time.  Results do not depend on the chunking: every
// plane is computed by the same per-site code whichever CTA owns it.
inline int z_chunks(int tiles, int planes, int per_sm, int fill) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    sms = (cudaGetDevice(&dev) == cudaSuccess &&
           cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) ? v : 152;
  }
  const long long slots = (long long)(per_sm > 0 ? per_sm : 1) * sms;
  int best_c = 1;
  long long best = -1;
  for (int c = 1; c <= planes && c <= 64; ++c) {
    const int zc = (planes + c - 1) / c;
    const long long waves = ((long long)tiles * c + slots - 1) / slots;
    const long long cost = waves * (zc + fill);
    if (best < 0 || cost < best) {
      best = cost;
      best_c = c;
    }
  }
  return best_c;
}

// CTAs of `kern` resident per SM at `threads` threads and `smem` bytes of dynamic shared memory
// (cached by the caller per kernel instantiation).
template <class K>
inline int resident_per_sm(K kern, int threads, size_t smem) {
  int v = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, threads, smem) != cudaSuccess || v < 1) {
    cudaGetLastError();
    v = 1;
  }
  return v;
}

template <class T, int ORDER, int S, int TX, int TYT, int RY, int P>
__global__ void __launch_bounds__(TX* TYT) k_stage3d_tma(const StageArgs<T> A, const __grid_constant__ CUtensorMap tm,
                                                        int zc, long long spin_limit, uint32_t extra_tx) {
  using C = typename T::C;
  using R = typename T::R;
  constexpr int TY = TYT * RY;   // rows of the tile; each thread computes RY of them
  using G = TmaGeom<TX, TY, C>;
  constexpr int RS = 5 + P;
  extern __shared__ __align__(128) unsigned char tma_smem[];
  unsigned char* slots = tma_smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(tma_smem + RS * G::kSlot);
  const Field<T>& f = A.f;
  const int nz = f.n[0], ny = f.n[1], nx = f.n[2];
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int zb = 1 + blockIdx.z * zc;
  const int ze = min(zb + zc, nz - 1);   // planes [zb, ze) are computed
  const int jb = zb - 2, jl = ze + 1;    // planes [jb, jl] are read
  const int64_t plane = (int64_t)ny * nx;
  const bool with_v = f.V != nullptr;

  if (tid == 0) {
    for (int s = 0; s < RS; ++s) mbar_init(smem_u32(bars + s), 1);
    mbar_fence_init();
  }
  __syncthreads();
  // slots are used round-robin: plane jb + q lives in slot q % RS
  int islot = 0;
  if (tid == 0) {
    for (int j = jb; j < jb + RS && j <= jl; ++j) {
      mbar_expect_tx(smem_u32(bars + islot), G::kBytes + extra_tx);
      tma_load_3d(smem_u32(slots + islot * G::kSlot), &tm, 2 * (x0 - 2), y0 - 2, j, smem_u32(bars + islot));
      islot = (islot + 1 == RS) ? 0 : islot + 1;
    }
  }
  int issued = min(jb + RS - 1, jl);

  const int gx = x0 + threadIdx.x;
  int gy[RY], o[RY];
  bool deep[RY];
  int64_t col[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    gy[r] = y0 + threadIdx.y + r * TYT;
    o[r] = (threadIdx.y + r * TYT + 2) * G::W + threadIdx.x + 2;
    // x, y at least 2 from the walls (x at least 2 + xwall when the slab shell owns more x layers)
    deep[r] = gx >= 2 + A.xwall && gx <= nx - 3 - A.xwall && gy[r] >= 2 && gy[r] <= ny - 3;
    col[r] = (int64_t)gy[r] * nx + gx;
  }

  // planes z-2 .. z+1 of the first plane
  const C* pl[5];
  int wslot = 0;
  uint32_t wpar = 0;
  bool late = false;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    late |= !mbar_wait_bounded(smem_u32(bars + wslot), wpar, spin_limit);
    pl[d] = reinterpret_cast<const C*>(slots + wslot * G::kSlot);
    if (++wslot == RS) { wslot = 0; wpar ^= 1u; }
  }

  PointVals<T> pv_next[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r)
    if (deep[r]) pv_next[r] = load_point<T, S>(A, zb * plane + col[r], with_v);
  bool aborted = false;
  for (int z = zb; z < ze; ++z) {
    PointVals<T> pv[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      pv[r] = pv_next[r];
      if (deep[r] && z + 1 < ze) pv_next[r] = load_point<T, S>(A, (z + 1) * plane + col[r], with_v);
    }
    late |= !mbar_wait_bounded(smem_u32(bars + wslot), wpar, spin_limit);
    pl[4] = reinterpret_cast<const C*>(slots + wslot * G::kSlot);
    if (++wslot == RS) { wslot = 0; wpar ^= 1u; }
    const bool deep_z = z >= 2 && z <= nz - 3;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      if (!(deep[r] && deep_z) || late) continue;   // wall-shell sites belong to the shell kernel
      const int idx[3] = {z, gy[r], gx};
      const int64_t c = z * plane + col[r];
      SAcc3<T> acc;
#pragma unroll
      for (int d = 0; d < 5; ++d) acc.p[d] = pl[d];
      acc.w = G::W;
      acc.o = o[r];
      const auto pc = acc.at0();
      const R Nc = fma(f.s, norm2(pc), -pv[r].v);
      const auto aL = a_lap_body<T, 3, ORDER, SAcc3<T>, false>(f, acc, idx, c, pc, Nc);
      rk_apply<T, S>(A, c, {-fma(Nc, pc.y, aL.y), fma(Nc, pc.x, aL.x)}, pv[r]);
    }
    if (__syncthreads_or(late)) {   // uniform decision: some copy never landed
      aborted = true;
      break;
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) pl[d] = pl[d + 1];
    if (tid == 0 && z - 2 + RS <= jl) {   // the slot of plane z-2 is free now
      mbar_expect_tx(smem_u32(bars + islot), G::kBytes + extra_tx);
      tma_load_3d(smem_u32(slots + islot * G::kSlot), &tm, 2 * (x0 - 2), y0 - 2, z - 2 + RS, smem_u32(bars + islot));
      islot = (islot + 1 == RS) ? 0 : islot + 1;
      issued = z - 2 + RS;
    }
  }
  if (aborted && tid == 0) {
    atomicOr(A.flag, kFlagTimeout);
    // the last RS planes issued are the only ones that can still be in flight
    for (int j = max(jb, issued - RS + 1); j <= issued; ++j) {
      const int q = j - jb;
      mbar_wait_bounded(smem_u32(bars + q % RS), uint32_t((q / RS) & 1), spin_limit);
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 exact-sum variant.  Each landed plane is converted once to fixed point
// (fix2) into a second ring that holds planes z-2 .. z+3, one plane ahead of
// use, so the per-plane barrier that releases slots also orders the
// conversion before the reads.  The FP64 ring only holds planes between
// their landing and their conversion (P + 1 slots); the centre values in
// FP64 come with the prefetched pointwise operands.  The stencil sums become
// exact integers; i2d_rn turns them into FP64 on the integer pipe.
// ---------------------------------------------------------------------------
template <class T, int ORDER, int S, int TX, int TYT, int RY, int P>
__global__ void __launch_bounds__(TX* TYT, 3) k_stage3d_tma_exact(const StageArgs<T> A,
                                                              const __grid_constant__ CUtensorMap tm, int zc,
                                                              long long spin_limit, uint32_t extra_tx) {
  static_assert(std::is_same<typename T::R, double>::value, "FP64 only");
  constexpr int TY = TYT * RY;
  using G = TmaGeom<TX, TY, double2>;
  constexpr int RD = P + 1;                        // FP64 landing slots
  constexpr int RF = 6;                            // fixed-point planes z-2 .. z+3
  constexpr int NT = TX * TYT, NPER = (G::PS + NT - 1) / NT;
  extern __shared__ __align__(128) unsigned char tma_smem[];
  unsigned char* dslots = tma_smem;
  longlong2* fring = reinterpret_cast<longlong2*>(tma_smem + RD * G::kSlot);
  uint64_t* bars = reinterpret_cast<uint64_t*>(tma_smem + (RD + RF) * G::kSlot);
  const Field<T>& f = A.f;
  const int nz = f.n[0], ny = f.n[1], nx = f.n[2];
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int zb = 1 + blockIdx.z * zc;
  const int ze = min(zb + zc, nz - 1);
  const int jb = zb - 2, jl = ze + 1;
  const int64_t plane = (int64_t)ny * nx;
  const bool with_v = f.V != nullptr;
  const int F = cur_fix(f), eadj = f.F - F;   // this step's fixed-point scale, and its shift to units of cLF
  unsigned int ex = 0;

  if (tid == 0) {
    for (int s = 0; s < RD; ++s) mbar_init(smem_u32(bars + s), 1);
    mbar_fence_init();
  }
  __syncthreads();
  int islot = 0, issued = jb - 1;
  auto issue = [&](int j) {
    mbar_expect_tx(smem_u32(bars + islot), G::kBytes + extra_tx);
    tma_load_3d(smem_u32(dslots + islot * G::kSlot), &tm, 2 * (x0 - 2), y0 - 2, j, smem_u32(bars + islot));
    islot = (islot + 1 == RD) ? 0 : islot + 1;
    issued = j;
  };
  if (tid == 0)
    for (int j = jb; j < jb + RD && j <= jl; ++j) issue(j);

  int wslot = 0, fslot = 0;
  uint32_t wpar = 0;
  bool late = false;
  // land plane j, convert it into the fixed ring; its FP64 slot is free after the next barrier
  auto land_and_convert = [&](int j) {
    late |= !mbar_wait_bounded(smem_u32(bars + wslot), wpar, spin_limit);
    const double2* src = reinterpret_cast<const double2*>(dslots + wslot * G::kSlot);
    longlong2* dst = fring + fslot * G::PS;
#pragma unroll
    for (int i = 0; i < NPER; ++i) {
      const int e = tid + i * NT;
      if (e < G::PS) dst[e] = fix2(src[e], F);
    }
    if (++wslot == RD) { wslot = 0; wpar ^= 1u; }
    fslot = (fslot + 1 == RF) ? 0 : fslot + 1;
  };

  const int gx = x0 + threadIdx.x;
  int gy[RY], o[RY];
  bool deep[RY];
  int64_t col[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    gy[r] = y0 + threadIdx.y + r * TYT;
    o[r] = (threadIdx.y + r * TYT + 2) * G::W + threadIdx.x + 2;
    deep[r] = gx >= 2 + A.xwall && gx <= nx - 3 - A.xwall && gy[r] >= 2 && gy[r] <= ny - 3;
    col[r] = (int64_t)gy[r] * nx + gx;
  }

  // planes jb .. jb+4 (z-2 .. z+2 of the first plane) into the fixed ring
  for (int j = jb; j <= jb + 4; ++j) {
    land_and_convert(j);
    __syncthreads();
    if (tid == 0 && issued < jl) issue(issued + 1);
  }
  int fz = 0;   // fixed slot of plane z-2

  PointVals<T> pv_next[RY];
  double2 pc_next[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r)
    if (deep[r]) {
      pv_next[r] = load_point<T, S, true>(A, zb * plane + col[r], with_v);
      pc_next[r] = f.in[zb * plane + col[r]];
    }
  bool aborted = false;
  for (int z = zb; z < ze; ++z) {
    PointVals<T> pv[RY];
    double2 pcs[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      pv[r] = pv_next[r];
      pcs[r] = pc_next[r];
      if (deep[r] && z + 1 < ze) {
        pv_next[r] = load_point<T, S, true>(A, (z + 1) * plane + col[r], with_v);
        pc_next[r] = f.in[(z + 1) * plane + col[r]];
      }
    }
    if (z + 3 <= jl) land_and_convert(z + 3);   // one plane ahead of use
    const bool deep_z = z >= 2 && z <= nz - 3;
    const longlong2* pl[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      const int q = fz + d;
      pl[d] = fring + (q >= RF ? q - RF : q) * G::PS;
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      if (!(deep[r] && deep_z) || late) continue;
      const int64_t c = z * plane + col[r];
      const int oo = o[r];
      const longlong2 cc = pl[2][oo];
      const longlong2 xm = pl[2][oo - 1], xp = pl[2][oo + 1], ym = pl[2][oo - G::W], yp = pl[2][oo + G::W];
      const longlong2 zm = pl[1][oo], zp = pl[3][oo];
      bool bad = fbad(cc) | fbad(xm) | fbad(xp) | fbad(ym) | fbad(yp) | fbad(zm) | fbad(zp);
      // axis order 0 (z), 1 (y), 2 (x) as in a_lap_exact
      long long s1x = (zp.x + zm.x) + (yp.x + ym.x) + (xp.x + xm.x);
      long long s1y = (zp.y + zm.y) + (yp.y + ym.y) + (xp.y + xm.y);
      long long Sx, Sy;
      if constexpr (ORDER == 2) {
        Sx = s1x - 6 * cc.x;
        Sy = s1y - 6 * cc.y;
      } else {
        const longlong2 xm2 = pl[2][oo - 2], xp2 = pl[2][oo + 2], ym2 = pl[2][oo - 2 * G::W],
                        yp2 = pl[2][oo + 2 * G::W], zm2 = pl[0][oo], zp2 = pl[4][oo];
        bad |= fbad(xm2) | fbad(xp2) | fbad(ym2) | fbad(yp2) | fbad(zm2) | fbad(zp2);
        const long long s2x = (zm2.x + zp2.x) + (ym2.x + yp2.x) + (xm2.x + xp2.x);
        const long long s2y = (zm2.y + zp2.y) + (ym2.y + yp2.y) + (xm2.y + xp2.y);
        Sx = 16 * s1x - s2x - 90 * cc.x;
        Sy = 16 * s1y - s2y - 90 * cc.y;
      }
      const double2 pc = pcs[r];
      // the exact-sum stages work in units of cLF: the integer sum needs no scaling, N_c is
      // formed from s / cLF and V / cLF, and the stage coefficients carry the cLF
      const double Nc = fma(f.sG, norm2(pc), -pv[r].v);
      double2 aL;
      if (!bad) {
        aL = {i2d_rn(Sx, eadj), i2d_rn(Sy, eadj)};
      } else {   // an operand out of the fixed-point range: the FP64 stencil from global memory
        const int idx[3] = {z, gy[r], gx};
        const GAcc<T, 3> ga(f, c);
        aL = a_lap_slow<T, 3, ORDER>(f, ga, idx, c, pc, Nc * f.cLF);
        aL = {aL.x * f.invcLF, aL.y * f.invcLF};
      }
      ex = max(ex, rk_apply<T, S>(A, c, {-fma(Nc, pc.y, aL.y), fma(Nc, pc.x, aL.x)}, pv[r]));
    }
    if (__syncthreads_or(late)) {
      aborted = true;
      break;
    }
    fz = (fz + 1 == RF) ? 0 : fz + 1;
    if (tid == 0 && issued < jl) issue(issued + 1);
  }
  if (S == 4 && A.emax) emax_commit(A.emax, ex);
  if (aborted && tid == 0) {
    atomicOr(A.flag, kFlagTimeout);
    for (int j = max(jb, issued - RD + 1); j <= issued; ++j) {
      const int q = j - jb;
      mbar_wait_bounded(smem_u32(bars + q % RD), uint32_t((q / RD) & 1), spin_limit);
    }
  }
}

template <class T, int ORDER, int S, int TX, int TYT, int RY, int P>
cudaError_t launch3d_tma_exact_shape(const StageArgs<T>& A, const CUtensorMap* tm, long long spin_limit,
                                     uint32_t extra_tx, cudaStream_t stream) {
  constexpr int TY = TYT * RY;
  using G = TmaGeom<TX, TY, double2>;
  const int nz = A.f.n[0], ny = A.f.n[1], nx = A.f.n[2];
  const int tiles = ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
  const int planes = nz - 2;
  const size_t smem = (P + 1 + 6) * G::kSlot + (P + 1) * sizeof(uint64_t);
  auto kern = k_stage3d_tma_exact<T, ORDER, S, TX, TYT, RY, P>;
  static int per_sm = 0;
  if (per_sm == 0) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    per_sm = resident_per_sm(kern, TX * TYT, smem);
  }
  int nzc = z_chunks(tiles, planes, per_sm, 4);
  const int zc = (planes + nzc - 1) / nzc;
  nzc = (planes + zc - 1) / zc;
  dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, nzc);
  kern<<<grid, dim3(TX, TYT), smem, stream>>>(A, *tm, zc, spin_limit, extra_tx);
  return cudaGetLastError();
}

template <class T, int ORDER, int S, int TX, int TYT, int RY, int P>
cudaError_t launch3d_tma_shape(const StageArgs<T>& A, const CUtensorMap* tm, long long spin_limit,
                               uint32_t extra_tx, cudaStream_t stream) {
  constexpr int TY = TYT * RY;
  using G = TmaGeom<TX, TY, typename T::C>;
  const int nz = A.f.n[0], ny = A.f.n[1], nx = A.f.n[2];
  const int tiles = ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
  const int planes = nz - 2;
  const size_t smem = (5 + P) * G::kSlot + (5 + P) * sizeof(uint64_t);
  auto kern = k_stage3d_tma<T, ORDER, S, TX, TYT, RY, P>;
  static int per_sm = 0;
  if (per_sm == 0) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    per_sm = resident_per_sm(kern, TX * TYT, smem);
  }
  int nzc = z_chunks(tiles, planes, per_sm, 4);
  const int zc = (planes + nzc - 1) / nzc;
  nzc = (planes + zc - 1) / zc;
  dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, nzc);
  kern<<<grid, dim3(TX, TYT), smem, stream>>>(A, *tm, zc, spin_limit, extra_tx);
  return cudaGetLastError();
}

template <class T, int ORDER, int S, bool EXACT>
cudaError_t launch3d_tma_stage(const StageArgs<T>& A, const LaunchCfg& L, cudaStream_t stream) {
  const CUtensorMap* tm = static_cast<const CUtensorMap*>(L.tmap);
  if constexpr (EXACT) {
    switch (L.tile_cfg) {
      case 1: return launch3d_tma_exact_shape<T, ORDER, S, 64, 4, 1, 2>(A, tm, L.spin_limit, L.extra_tx, stream);
      case 2: return launch3d_tma_exact_shape<T, ORDER, S, 32, 8, 2, 2>(A, tm, L.spin_limit, L.extra_tx, stream);
      case 3: return launch3d_tma_exact_shape<T, ORDER, S, 64, 4, 2, 2>(A, tm, L.spin_limit, L.extra_tx, stream);
      default: return launch3d_tma_exact_shape<T, ORDER, S, 32, 8, 1, 2>(A, tm, L.spin_limit, L.extra_tx, stream);
    }
  } else {
    switch (L.tile_cfg) {   // the tile shapes of tma_tile_shape()
      case 1: return launch3d_tma_shape<T, ORDER, S, 64, 4, 1, 2>(A, tm, L.spin_limit, L.extra_tx, stream);
      case 2: return launch3d_tma_shape<T, ORDER, S, 32, 8, 2, 2>(A, tm, L.spin_limit, L.extra_tx, stream);
      case 3: return launch3d_tma_shape<T, ORDER, S, 64, 4, 2, 2>(A, tm, L.spin_limit, L.extra_tx, stream);
      default: return launch3d_tma_shape<T, ORDER, S, 32, 8, 1, 2>(A, tm, L.spin_limit, L.extra_tx, stream);
    }
  }
}

template <class T, int ORDER, bool EXACT>
cudaError_t launch3d_tma(const StageArgs<T>& A, const LaunchCfg& L, cudaStream_t stream) {
  switch (A.stage) {
    case 1: return launch3d_tma_stage<T, ORDER, 1, EXACT>(A, L, stream);
    case 2: return launch3d_tma_stage<T, ORDER, 2, EXACT>(A, L, stream);
    case 3: return launch3d_tma_stage<T, ORDER, 3, EXACT>(A, L, stream);
    default: return launch3d_tma_stage<T, ORDER, 4, EXACT>(A, L, stream);
  }
}

}  // namespace nlse
