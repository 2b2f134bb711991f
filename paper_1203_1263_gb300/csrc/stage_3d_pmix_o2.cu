// 3D stage launches for PMix, order 2 (see stage_3d_impl.cuh).
#include "stage_3d_impl.cuh"

namespace nlse {
template cudaError_t launch_stage<PMix, 3, 2>(const StageArgs<PMix>&, const LaunchCfg&, cudaStream_t);
}  // namespace nlse
