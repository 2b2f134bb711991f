// 3D stage launches: variant 0 = generic kernel, 1 = z-marching tiled kernel
// (TMA-fed when the layout allows, else cooperative loads),
// 2 / 3 = tiled / generic with the exact-sum stencil (FP64 only).
// Included by one small translation unit per (precision, order), so that the
// many kernel instantiations compile in parallel.
#pragma once
#include "stage_generic.cuh"
#include "stage_slab.cuh"
#include "stage_tiled.cuh"
#include "stage_tma.cuh"

namespace nlse {

template <class T, int D, int ORDER>
cudaError_t launch_stage(const StageArgs<T>& A, const LaunchCfg& L, cudaStream_t stream) {
  constexpr bool fp64 = std::is_same<typename T::R, double>::value;
  const int variant = (!fp64 && L.variant >= 2) ? L.variant - 2 : L.variant;   // exact sums are FP64 only
  const bool exact = variant >= 2;
  const bool periodic = A.f.bc == BC_PERIODIC;
  if (variant == 0 || variant == 3) {
    if (periodic) {
      if constexpr (fp64) if (exact) return launch_generic_periodic<T, D, ORDER, true>(A, stream);
      return launch_generic_periodic<T, D, ORDER>(A, stream);
    }
    if constexpr (fp64) if (exact) return launch_generic<T, D, ORDER, true>(A, stream);
    return launch_generic<T, D, ORDER>(A, stream);
  }
  // tiled: deep interior (TMA-fed when the layout allows) + the wall shell, as
  // shared-memory slabs (FP32 stages: three x layers per x wall) or, for thin
  // grids and periodic grids (whose shell wraps), the global-memory shell kernel
  const bool slabs = slab_ok(A.f.n) && !periodic;
  constexpr int nsx = fp64 ? 1 : 3;   // x-wall layers owned by the slab shell
  StageArgs<T> B = A;
  B.xwall = slabs ? nsx - 1 : 0;
  auto deep = [&](cudaStream_t st) -> cudaError_t {
    if constexpr (fp64) {
      if (exact) return L.tmap ? launch3d_tma<T, ORDER, true>(B, L, st) : launch3d_tiled<T, ORDER, true>(B, L.tile_cfg, st);
    }
    return L.tmap ? launch3d_tma<T, ORDER, false>(B, L, st) : launch3d_tiled<T, ORDER>(B, L.tile_cfg, st);
  };
  auto shell = [&](cudaStream_t st) -> cudaError_t {
    if (periodic) {
      if constexpr (fp64) if (exact) return launch_shell_periodic<T, D, ORDER, true>(B, st);
      return launch_shell_periodic<T, D, ORDER>(B, st);
    }
    if (slabs) {
      if constexpr (fp64) if (exact) return launch_shell_slabs<T, ORDER, true, nsx>(B, st, L.side_yx);
      return launch_shell_slabs<T, ORDER, false, nsx>(B, st, L.side_yx);
    }
    if constexpr (fp64) if (exact) return launch_shell<T, D, ORDER, true>(B, st);
    return launch_shell<T, D, ORDER>(B, st);
  };
  if (slabs) return launch_deep_and_shell(L, stream, has_deep(D, A.f.m), deep, shell);
  LaunchCfg L1 = L;   // one shell kernel: no use for the slabs' extra streams
  L1.side_yx[0] = L1.side_yx[1] = nullptr;
  return launch_deep_and_shell(L1, stream, has_deep(D, A.f.m), deep, shell);
}

}  // namespace nlse
