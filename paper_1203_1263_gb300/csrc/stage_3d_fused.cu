// The FP32 form's two-stages-per-pass RK4 step on 3D grids (stage_fused.cuh):
// per pass, the first stage's wall shell (slab kernels, on the side stream)
// runs concurrently with the fused deep kernel, then the second stage's shell.
#include "stage_fused.cuh"

namespace nlse {

template <int ORDER>
cudaError_t launch_fused_step(const StageArgs<P32>* A, const void* tm12, const void* tm34, const LaunchCfg& L,
                              cudaStream_t stream) {
  for (int pass = 0; pass < 2; ++pass) {
    const StageArgs<P32>& A1 = A[2 * pass];
    const StageArgs<P32>& A2 = A[2 * pass + 1];
    StageArgs<P32> B1 = A1;
    B1.xwall = 2;   // the first stage's shell owns x = 1..3 and its mirror
    const CUtensorMap* tm = static_cast<const CUtensorMap*>(pass == 0 ? tm12 : tm34);
    auto deep = [&](cudaStream_t st) -> cudaError_t {
      return pass == 0 ? launch_fused_kernel<ORDER, 1>(A1, A2, tm, L.spin_limit, L.extra_tx, st)
                       : launch_fused_kernel<ORDER, 3>(A1, A2, tm, L.spin_limit, L.extra_tx, st);
    };
    auto shell = [&](cudaStream_t st) -> cudaError_t { return launch_shell_slabs<P32, ORDER, false, 3>(B1, st, L.side_yx); };
    cudaError_t e = launch_deep_and_shell(L, stream, true, deep, shell);
    if (e != cudaSuccess) return e;
    if ((e = launch_shell_slabs3<ORDER>(A2, stream)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template cudaError_t launch_fused_step<2>(const StageArgs<P32>*, const void*, const void*, const LaunchCfg&, cudaStream_t);
template cudaError_t launch_fused_step<4>(const StageArgs<P32>*, const void*, const void*, const LaunchCfg&, cudaStream_t);

bool fused_grid_ok(int d, const int* n) { return d == 3 && fused_ok(n); }

}  // namespace nlse
