// 2D stage launches: variant 0 = generic kernel, 1 = halo-tiled kernel,
// 2 / 3 = tiled / generic with the exact-sum stencil (FP64 only).
#include "stage_generic.cuh"
#include "stage_tiled.cuh"

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
  // tiled: deep interior + the wall shell (periodic grids: the two layers at each end of each axis)
  auto deep = [&](cudaStream_t st) -> cudaError_t {
    if constexpr (fp64) if (exact) return launch2d_tiled<T, ORDER, true>(A, L.tile_cfg, st);
    return launch2d_tiled<T, ORDER>(A, L.tile_cfg, st);
  };
  auto shell = [&](cudaStream_t st) -> cudaError_t {
    if (periodic) {
      if constexpr (fp64) if (exact) return launch_shell_periodic<T, D, ORDER, true>(A, st);
      return launch_shell_periodic<T, D, ORDER>(A, st);
    }
    if constexpr (fp64) if (exact) return launch_shell<T, D, ORDER, true>(A, st);
    return launch_shell<T, D, ORDER>(A, st);
  };
  return launch_deep_and_shell(L, stream, has_deep(D, A.f.m), deep, shell);
}

#define INST(T, O) template cudaError_t launch_stage<T, 2, O>(const StageArgs<T>&, const LaunchCfg&, cudaStream_t);
INST(P64, 2) INST(P64, 4) INST(P32, 2) INST(P32, 4) INST(PMix, 2) INST(PMix, 4)
#undef INST

}  // namespace nlse
