// 3D stage launches for P64, order 4 (see stage_3d_impl.cuh).
#include "stage_3d_impl.cuh"

namespace nlse {
template cudaError_t launch_stage<P64, 3, 4>(const StageArgs<P64>&, const LaunchCfg&, cudaStream_t);
}  // namespace nlse
