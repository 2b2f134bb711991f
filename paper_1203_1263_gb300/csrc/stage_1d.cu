// 1D stage launches: the generic kernel; whole calls of nsteps steps on one
// thread-block cluster (stage_line1d.cuh).
#include "stage_generic.cuh"
#include "stage_line1d.cuh"
#include "nlse_internal.h"

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

bool line_ok(int n, bool fp64) {
  int cl, seg;
  size_t smem;
  return line_plan(n, fp64 ? 16 : 8, &cl, &seg, &smem);
}

template <class T>
cudaError_t launch_line_steps(const StageArgs<T>* A, int64_t nsteps, int n, int order, bool exact, int F0,
                              int fix_offset, cudaStream_t stream) {
  int cl, seg;
  size_t smem;
  if (!line_plan(n, sizeof(typename T::C), &cl, &seg, &smem)) return cudaErrorInvalidConfiguration;
  LineArgs<T> L;
  memset(&L, 0, sizeof(L));
  for (int s = 0; s < 4; ++s) L.A[s] = A[s];
  L.nsteps = nsteps;
  L.n = n;
  L.seg = seg;
  L.F0 = F0;
  L.fix_offset = fix_offset;
  if constexpr (std::is_same<T, P64>::value) {
    if (exact)
      return order == 4 ? launch_line1d<T, 4, true>(L, cl, smem, stream) : launch_line1d<T, 2, true>(L, cl, smem, stream);
  }
  return order == 4 ? launch_line1d<T, 4, false>(L, cl, smem, stream) : launch_line1d<T, 2, false>(L, cl, smem, stream);
}

template cudaError_t launch_line_steps<P64>(const StageArgs<P64>*, int64_t, int, int, bool, int, int, cudaStream_t);
template cudaError_t launch_line_steps<P32>(const StageArgs<P32>*, int64_t, int, int, bool, int, int, cudaStream_t);

}  // namespace nlse
