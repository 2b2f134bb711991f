// Launchers shared between the library's translation units (not exported).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "nlse_device.cuh"

namespace nlse {

constexpr int kMaxReduceBlocks = 1024;

// CTA tile (x-by-y threads) of the tiled 3D/2D kernels for tile_cfg 0..3.
inline void tma_tile_shape(int tile_cfg, int* tx, int* ty) {
  switch (tile_cfg) {
    case 1: *tx = 64; *ty = 4; break;
    case 2: *tx = 32; *ty = 16; break;
    case 3: *tx = 64; *ty = 8; break;
    default: *tx = 32; *ty = 8; break;
  }
}

// The FP32 form's fused step (two RK4 stages per pass; stage_fused.cuh): A[0..3]
// are stages 1..4, tm12 / tm34 the TMA descriptors of the passes' inputs
// (Psi^n, Psi_out) with the fused kernel's box (fused_box below).
template <int ORDER>
cudaError_t launch_fused_step(const StageArgs<P32>* A, const void* tm12, const void* tm34, const LaunchCfg& L,
                              cudaStream_t stream);
bool fused_grid_ok(int d, const int* n);
// the fused kernel's TMA box: 64 + 8 complex values by 8 + 8 rows
constexpr int kFusedBoxX = 2 * (64 + 8), kFusedBoxY = 8 + 8;

// 1D lines on one thread-block cluster (stage_line1d.cuh): nsteps RK4 steps of
// an n-site line in one launch; A[0..3] are stages 1..4 with Psi updated in
// place.  cudaErrorInvalidConfiguration when the line does not fit or the
// cluster cannot be co-scheduled (the caller then takes the per-site kernel).
bool line_ok(int n, bool fp64);
template <class T>
cudaError_t launch_line_steps(const StageArgs<T>* A, int64_t nsteps, int n, int order, bool exact, int F0,
                              int fix_offset, cudaStream_t stream);

cudaError_t launch_mass(const void* psi, bool psi_double, int64_t total, double scale, double* partials,
                        double* result, unsigned int* flag, cudaStream_t stream);
template <class T, int D, int ORDER>
cudaError_t launch_energy(const Field<T>& f, double scale, double* partials, double* result, unsigned int* flag,
                          cudaStream_t stream);
cudaError_t launch_vmax(const void* V, bool v_double, int64_t total, unsigned long long* out, cudaStream_t stream);
// Exact-sum scale: with psi (complex128, n = 2 x sites components) first the
// largest exponent of psi into *emax, then *fdev = the fraction bits for it
// (+ offset) and *emax = 0.  With psi == nullptr only the second part (the
// exponent was collected by the stage-4 kernels).
cudaError_t launch_fix_update(const double* psi, int64_t n, unsigned int* emax, int* fdev, int F0, int offset,
                              cudaStream_t stream);
cudaError_t launch_round_master(const double2* master, float2* n32, int64_t total, cudaStream_t stream);
cudaError_t launch_scale_v(const double* V, double s, int64_t n, double* Vs, cudaStream_t stream);

}  // namespace nlse
