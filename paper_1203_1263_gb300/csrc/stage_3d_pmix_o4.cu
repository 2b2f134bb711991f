// 3D stage launches for PMix, order 4 (see stage_3d_impl.cuh).
#include "stage_3d_impl.cuh"

namespace nlse {
template cudaError_t launch_stage<PMix, 3, 4>(const StageArgs<PMix>&, const LaunchCfg&, cudaStream_t);
}  // namespace nlse
