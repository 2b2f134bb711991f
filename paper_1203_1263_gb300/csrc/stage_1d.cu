// 1D stage launches: the generic kernel.
#include "stage_generic.cuh"

namespace nlse {

template <class T, int D, int ORDER>
cudaError_t launch_stage(const StageArgs<T>& A, int variant, int tile_cfg, cudaStream_t stream) {
  (void)variant; (void)tile_cfg;
  return launch_generic<T, D, ORDER>(A, stream);
}

#define INST(T, O) template cudaError_t launch_stage<T, 1, O>(const StageArgs<T>&, int, int, cudaStream_t);
INST(P64, 2) INST(P64, 4) INST(P32, 2) INST(P32, 4) INST(PMix, 2) INST(PMix, 4)
#undef INST

}  // namespace nlse
