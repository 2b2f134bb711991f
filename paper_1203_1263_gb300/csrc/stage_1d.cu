// 1D stage launches: the generic kernel.
#include "stage_generic.cuh"

namespace nlse {

template <class T, int D, int ORDER>
cudaError_t launch_stage(const StageArgs<T>& A, const LaunchCfg& L, cudaStream_t stream) {
  const int variant = L.variant, tile_cfg = L.tile_cfg;
  (void)tile_cfg;
  const bool periodic = A.f.bc == BC_PERIODIC;
  if constexpr (std::is_same<typename T::R, double>::value) {
    if (variant >= 2)
      return periodic ? launch_generic_periodic<T, D, ORDER, true>(A, stream) : launch_generic<T, D, ORDER, true>(A, stream);
  }
  return periodic ? launch_generic_periodic<T, D, ORDER>(A, stream) : launch_generic<T, D, ORDER>(A, stream);
}

#define INST(T, O) template cudaError_t launch_stage<T, 1, O>(const StageArgs<T>&, const LaunchCfg&, cudaStream_t);
INST(P64, 2) INST(P64, 4) INST(P32, 2) INST(P32, 4) INST(PMix, 2) INST(PMix, 4)
#undef INST

}  // namespace nlse
