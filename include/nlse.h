/*
 * nlse.h -- C ABI of the GB300 (sm_103a) RK4 integrator for the nonlinear
 * Schroedinger / Gross-Pitaevskii equation
 *
 *     i dPsi/dt + a Lap(Psi) - V(r) Psi + s |Psi|^2 Psi = 0          (Sec. 1, Eq. NLSE)
 *
 * on 1D, 2D and 3D complex grids with one spacing h on every axis (Sec. 3,
 * Eq. disc), advanced by classic RK4 (Sec. 3.1, Eq. RK4) with F(Psi) =
 * i[a Lap Psi + (s|Psi|^2 - V) Psi], the central-difference (order 2) or
 * two-step compact 2SHOC (order 4) Laplacian (Sec. 3.2), and the Dirichlet
 * or modulus-squared Dirichlet (MSD) boundary (Sec. 3.3).
 *
 * Conventions shared by every call
 *   Layout     C order, last index fastest: a 3D grid is (N[0], N[1], N[2]) =
 *              (Nz, Ny, Nx).  Boundary sites are those with any index 0 or
 *              N[k]-1; the rest are interior (a periodic grid has no
 *              boundary sites).  Every N[k] >= 3.
 *   Psi        interleaved complex: NLSE_C128 -> double2 (re, im),
 *              NLSE_C64 -> float2, NLSE_C64_ACC64 -> double2 (the FP64 master).
 *   V          real, same shape: double for NLSE_C128, float for the other two;
 *              NULL means V = 0.  The library reads V when a context is
 *              created and when nlse_refresh_potential is called: every dtype
 *              takes max|V| for the stability check from those reads, and
 *              NLSE_C128 integrates with a scaled copy of V made there (the
 *              FP32 forms read V itself).  After writing new values into V,
 *              call nlse_refresh_potential before the next nlse_step.
 *   Pointers   psi, V and workspace are DEVICE pointers owned by the caller.
 *              The library never allocates, frees or copies them; a context
 *              borrows them until nlse_destroy.  Host pointers are named *_host.
 *   Streams    stream is a cudaStream_t passed as void* (NULL = legacy default
 *              stream).  nlse_step is asynchronous on that stream; nlse_mass,
 *              nlse_energy and nlse_sync synchronise it.
 *   Errors     every int-returning call returns NLSE_OK (0) or a negative
 *              status below; nlse_last_error() gives a message for the last
 *              failure on the calling thread.  A failed call changes nothing
 *              unless its description says otherwise.
 */
#ifndef NLSE_H
#define NLSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define NLSE_OK          0
#define NLSE_EINVAL     -1  /* bad argument (dims, N, h, a, order, bc, dtype, pointer, dt <= 0) */
#define NLSE_ENOMEM     -2  /* the caller's workspace is smaller than nlse_workspace_bytes() */
#define NLSE_ECUDA      -3  /* a CUDA launch or runtime call failed */
#define NLSE_EUNSTABLE  -4  /* dt above the RK4 linear stability bound (see nlse_max_dt) */
#define NLSE_ENONFINITE -5  /* a NaN or Inf appeared in Psi (sticky until the next nlse_create) */
#define NLSE_ETIMEOUT   -6  /* a bounded device-side wait gave up */
#define NLSE_ESTATE     -7  /* call not valid in the context's current state */

/* ---- boundary conditions (Sec. 3.3) ---- */
#define NLSE_BC_DIRICHLET 0 /* Eq. BCDdef: Psi_b is held at its value; Laplacian form Eq. BCDlap */
#define NLSE_BC_MSD       1 /* Eq. BCMSDdef: |Psi_b|^2 held; Eq. msd and Eq. BCMSDlap */
#define NLSE_BC_L0        2 /* Laplacian-zero: dPsi_b/dt = i(s|Psi_b|^2 - V_b) Psi_b (Eq. BCL0dt),
                               Laplacian form D_b = 0 (Eq. BCL0lap) */
#define NLSE_BC_PERIODIC  3 /* periodic grid, the boundary the RK4 stability analysis of Sec. 3.4
                               assumes (not one of the paper's wall forms): no boundary sites, site
                               N[k] along axis k is site 0 again (period N[k] h), every site is
                               updated; mass and energy sum over every site.  Not available in the
                               batched form. */

/* ---- precision forms ---- */
#define NLSE_C128      0 /* FP64 throughout */
#define NLSE_C64       1 /* FP32 throughout (the paper's single-precision codes, Sec. 5.2) */
#define NLSE_C64_ACC64 2 /* FP32 stage arithmetic and stage arrays, FP64 master Psi and RK4
                            accumulation (Psi^{n+1} = Psi^n + dt/6 (K_tot + k) in FP64),
                            FP64 mass/energy reductions */

typedef struct nlse_ctx *nlse_t;

/*
 * Bytes of device workspace a context needs (stage arrays K_tot, Psi_tmp,
 * Psi_out of Eq. RK4_GPU in the dtype's stage precision, plus the FP32 copy
 * of Psi^n for NLSE_C64_ACC64, reduction partials and status words).
 * Returns 0 for invalid arguments.
 */
size_t nlse_workspace_bytes(int dims, const int64_t *N, int dtype);

/*
 * Create an integrator context over caller-owned device memory.
 *   dims       1, 2 or 3;  N: host array of dims extents, each >= 3
 *   h, a       grid spacing and dispersion coefficient, both > 0;  s: any real
 *   V          device potential (see conventions) or NULL
 *   bc, order  NLSE_BC_*, and 2 (central difference) or 4 (2SHOC)
 *   psi        device Psi, read and written in place by nlse_step
 *   workspace  device buffer of at least nlse_workspace_bytes(), 256-byte aligned
 *   stream     cudaStream_t for every launch of this context
 * Synchronises the stream once (it measures max|V| for the stability check).
 * On success *out receives the context.
 */
int nlse_create(nlse_t *out, int dims, const int64_t *N, double h, double a, double s, const void *V, int bc,
                int order, int dtype, void *psi, void *workspace, size_t ws_bytes, void *stream);

/*
 * Re-read the context's potential V after the caller wrote new values into
 * it: max|V| for the stability check and, for NLSE_C128, the scaled copy the
 * exact-sum stages integrate with.  Synchronises the stream once (when V is
 * not NULL).  NLSE_ECUDA on a CUDA failure.
 */
int nlse_refresh_potential(nlse_t ctx);

/*
 * Advance Psi by nsteps RK4 steps of size dt (Eq. RK4, computed as the four
 * fused stages of Eq. RK4_GPU: each stage evaluates F with the boundary
 * condition and applies its update in one pass).  Asynchronous on the
 * context's stream.  nsteps == 0 is a no-op.  Fails with NLSE_EUNSTABLE when
 * dt exceeds nlse_max_dt(dims, h, a, order, max|V|, 0), the linear bound
 * without the 0.8 safety factor the paper's drivers apply.  Calling it twice
 * with n1 and n2 steps gives bit-for-bit the result of one call with n1 + n2.
 */
int nlse_step(nlse_t ctx, int64_t nsteps, double dt);

/*
 * Mass  M = h^d sum_{all sites} |Psi|^2, in FP64 with compensated
 * (Neumaier) summation and a deterministic two-pass reduction.  Synchronises
 * the stream.  Returns NLSE_ENONFINITE if Psi holds a NaN or Inf.
 */
int nlse_mass(nlse_t ctx, double *out_host);

/*
 * Energy  E = h^d sum_{interior} [ -a Re(conj(Psi) Lap Psi) + V|Psi|^2 - (s/2)|Psi|^4 ]
 * with the context's own Laplacian (order and boundary Laplacian form), in
 * FP64.  The paper defines no energy; this is the discrete Hamiltonian of the
 * semi-discrete flow.  Synchronises the stream.
 */
int nlse_energy(nlse_t ctx, double *out_host);

/*
 * F(Psi) = i[a Lap Psi + (s|Psi|^2 - V) Psi] at every site of an arbitrary
 * state psi_in (same dtype, shape and device as the context's Psi; for
 * NLSE_C64_ACC64 it is float2), written to F_out (same type).  Boundary sites
 * get the boundary condition's time derivative (Eqs. BCDdt, msd).
 * Asynchronous.  For testing the right-hand side on its own.
 */
int nlse_rhs(nlse_t ctx, const void *psi_in, void *F_out);

/*
 * RK4 linear stability bound on dt (Sec. 3.4): 2 sqrt(2) / (a rho_L + vmax +
 * s_rho_max) with rho_L = 4d/h^2 (order 2) or 16d/(3h^2) (order 4).  With
 * vmax = s_rho_max = 0 this is Eqs. stblincd / stblin2shoc.  Drivers usually
 * take 0.8 of it.  Returns a negative value for invalid arguments.
 */
double nlse_max_dt(int dims, double h, double a, int order, double vmax, double s_rho_max);

/* Wait for the context's stream and report a sticky non-finite flag or a
 * CUDA error. */
int nlse_sync(nlse_t ctx);

/* Release the context (never the caller's device buffers). */
int nlse_destroy(nlse_t ctx);

/* Message for the last failed call on this thread ("" if none). */
const char *nlse_last_error(void);

/* Which stage kernel the context uses:
 *   0 = generic one-thread-per-site kernel,
 *   1 = tiled kernel (2D halo tiles / 3D z-marching; on 1D lines of up to
 *       ~49,000 sites in FP64 or ~98,000 in FP32 (not NLSE_C64_ACC64) one
 *       thread-block cluster of up to 16 CTAs keeps the line in shared memory
 *       and runs every step of an nlse_step call in one launch; longer lines
 *       and the mixed form use the generic kernel),
 *   2 = tiled kernel with the exact-sum stencil (NLSE_C128 only; other
 *       dtypes treat it as 1): the Laplacian's stencil sums are formed exactly
 *       in 64-bit fixed point on the integer pipe and converted to FP64 once,
 *   3 = generic kernel with the exact-sum stencil (NLSE_C128; else as 0).
 * Variants 0 and 1 give bit-for-bit the same result, and so do 2 and 3.
 * Default: 2 for NLSE_C128 and 1 otherwise, except on grids small enough
 * that a step is bound by latency rather than by throughput: 3D grids of at
 * most 2^15 sites (NLSE_C128) or 2^17 sites (the FP32 forms) take 0,
 * NLSE_C128 2D grids of at most 80,000 sites take 1, and NLSE_C128 1D lines
 * take 1 (the cluster path) up to 2500 sites, 0 up to 2^15 sites and 3
 * beyond (the plain FP64 stencil's instruction chain is shorter than the
 * exact-sum stencil's conversions; a cluster's 16 SMs bound longer lines).
 * The exact-sum stencil's fixed-point scale follows the state: before every
 * step it is taken from the largest component of Psi (every component
 * below 2^53 in fixed point, 4x below the accepted range, so the largest
 * components keep all 53 bits), at the start of each nlse_step from a pass
 * over Psi (the caller may have written it) and after each step from the
 * values the step wrote; a site whose operand is still out of range (a
 * stage state more than 4x the step's largest component) takes the FP64
 * stencil.  The resolution is thus 2^-52 or finer relative to max|Psi| for
 * any state, and results never depend on how steps are split into calls.
 *   4 = NLSE_C64 on 3D grids: two RK4 stages per pass (stages 1+2 and 3+4,
 *       temporal blocking): the first stage's result for a tile plus a
 *       two-cell halo stays on chip and feeds the second stage, so the
 *       intermediate state never goes through HBM (about 64 instead of 152
 *       bytes per interior site and step); it applies to the 16-step chunks
 *       nlse_step replays as CUDA graphs on grids with every extent >= 16,
 *       an even Nx and a wall boundary, and Psi alternates with a copy in the
 *       workspace inside each chunk (the chunk ends in Psi).  Other steps,
 *       dtypes and grids run as 1.  Same results as 1, bit for bit.
 * tile_cfg picks the tiled kernel's CTA tile (x-by-y threads): 0 = 32x8,
 * 1 = 64x4, 2 = 32x16, 3 = 64x8, -1 = default; it never changes results.
 * Call between nlse_step calls, not during one. */
int nlse_set_kernel(nlse_t ctx, int variant, int tile_cfg);

/* The stage kernel variant nlse_step's graph-replayed steps run with, after
 * the context's grid, dtype and boundary are taken into account (0..4 as in
 * nlse_set_kernel), or a negative status. */
int nlse_kernel_in_use(nlse_t ctx);

/*
 * Autotuner: time every tile shape of the context's tiled kernel on its own
 * buffers (stage 1 then repeated stage-2 launches; Psi is read, never
 * written) and keep the fastest for this context.  The choice is cached for
 * the process per (dims, shape, dtype, order, bc, variant, V present), and
 * appended to the text file named by the environment variable
 * NLSE_TUNE_CACHE when it is set (later processes read it instead of
 * timing).  Synchronises the stream.  *best_tile_cfg receives the chosen
 * tile_cfg (-1 when nothing is tiled: 1D grids, variants 0 and 3) and
 * *best_ms the measured stage-2 time (0 when taken from a cache); either
 * pointer may be NULL.  Tiles never change results.
 */
int nlse_autotune(nlse_t ctx, int *best_tile_cfg, float *best_ms);

/* ---------------------------------------------------------------------------
 * Batched form: many independent 2D runs (uneven sizes and parameters) in
 * complex64, advanced together with one launch per RK4 stage for all runs
 * (a persistent deep-interior kernel over a (run, tile) work list and a
 * wall-shell kernel over the runs' walls), the step loop replayed as a CUDA
 * graph.  Each run is computed with the same per-site arithmetic as a
 * single-run NLSE_C64 context with the tiled kernel, so its result is
 * bit-for-bit that of integrating it alone.
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t n[2];        /* (Ny, Nx), each >= 3 */
  double h, a, s, dt;  /* spacing, dispersion, nonlinearity, this run's time step */
  int bc, order;       /* NLSE_BC_*, 2 or 4 */
  void *psi;           /* device complex64 (float2), caller-owned, advanced in place */
  const void *V;       /* device float32 potential of the run's shape, or NULL */
} nlse_run_desc;

typedef struct nlse_batch *nlse_batch_t;

/* Workspace bytes for the runs (per-run stage arrays, run table, work lists);
 * 0 for invalid descriptors. */
size_t nlse_batch_workspace_bytes(int nruns, const nlse_run_desc *runs);

/* Create a batch over caller-owned device memory (descriptors are copied).
 * Fails with NLSE_EUNSTABLE when a run's dt exceeds its RK4 linear bound
 * (Sec. 3.4 with V = s = 0).  Synchronises the stream once (table upload). */
int nlse_batch_create(nlse_batch_t *out, int nruns, const nlse_run_desc *runs, void *workspace, size_t ws_bytes,
                      void *stream);

/* Advance every run by nsteps RK4 steps of its own dt; asynchronous. */
int nlse_batch_step(nlse_batch_t b, int64_t nsteps);

/* Tile shape of the batched deep kernel (as nlse_set_kernel's tile_cfg; -1 = 32x8, the measured best on
 * the 512-run workload). */
int nlse_batch_set_tile(nlse_batch_t b, int tile_cfg);

/* Autotuner: time stages 1-3 of every tile shape on the batch's own runs
 * (three passes in alternating order, the first one untimed; none of these
 * stages writes any run's Psi) and keep the fastest shape; *best_ms is its
 * mean stage time.  Synchronises the stream. */
int nlse_batch_autotune(nlse_batch_t b, int *best_tile_cfg, float *best_ms);

/* Wait for the stream; NLSE_ENONFINITE if any run produced a NaN or Inf. */
int nlse_batch_sync(nlse_batch_t b);

int nlse_batch_destroy(nlse_batch_t b);

/* ---------------------------------------------------------------------------
 * Learned surrogate (not in the paper): a residual 3x3-convolution network
 * that maps a 2D complex64 state psi(t) to psi(t + window), trained on states
 * the integrator itself produced.
 *   h_{-1} = (Re psi, Im psi, |psi|^2 Re psi, |psi|^2 Im psi)  (the cubic term as input features);
 *   z_l = conv3x3_{dil_l}(h_{l-1}) + b_l,  h_l = silu(z_l)
 *   (l = 0 .. layers-2, `channels` channels);  y = conv3x3(h_{layers-2}) + b (2 channels);
 *   psi_out = psi_in + (y_0 + i y_1);  zero padding at the grid edges.
 * Loss: the mean squared error of psi_out's real and imaginary parts, plus
 * mass_weight (nlse_sur_set_mass_weight; 0 by default) times the mean over
 * the batch's states of ((M(psi_out) - M(target)) / M(target))^2 with
 * M = sum |psi|^2 over the state: the NLSE conserves mass, and the term
 * teaches the network to conserve it without the projection below.
 * Activations are channels-last; every convolution (forward, backward-data,
 * weight-gradient) is an implicit GEMM on the tensor cores with BF16 operands
 * and FP32 accumulation; parameters are FP32 masters (layout per layer: W
 * [cout][9][cin] then b [cout]) with BF16 copies; optimiser Adam (0.9, 0.999, 1e-8).
 * All pointers are device pointers owned by the caller; states are float2
 * arrays [nb][H][W].  Asynchronous unless a host output is requested.
 * ------------------------------------------------------------------------- */
typedef struct nlse_sur *nlse_sur_t;

/* Number of FP32 parameters (0 for invalid shapes: channels 1..256, layers 2..16). */
size_t nlse_sur_param_count(int channels, int layers);

/* Workspace bytes for batches of up to max_batch states of H x W. */
size_t nlse_sur_workspace_bytes(int H, int W, int channels, int layers, int max_batch);

/* Create over caller-owned params (nlse_sur_param_count floats) and workspace. */
int nlse_sur_create(nlse_sur_t *out, int H, int W, int channels, int layers, const int *dilations, int max_batch,
                    float *params, void *workspace, size_t ws_bytes, void *stream);

/* Seeded uniform initialisation of the parameters (SplitMix64), Adam state reset. */
int nlse_sur_init(nlse_sur_t s, uint64_t seed);

/* Refresh the BF16 copies after the caller wrote params directly. */
int nlse_sur_sync_params(nlse_sur_t s);

/* psi_out = network(psi_in) for nb states (nb <= max_batch).  With
 * masses_out (device, 2 nb doubles; NULL to skip) state b's sums
 * M(psi_in) = sum |psi_in|^2 and M(raw) = sum |psi_out|^2 of the network's
 * output as it came out, before any projection, go to masses_out[2b] and
 * masses_out[2b + 1] (FP64, fixed summation order): the raw output's mass is
 * what a caller judges the network's mass conservation by.  With
 * project_mass != 0 each output state is then rescaled by
 * sqrt(M(psi_in) / M(raw)), so that it carries its input's mass, which the
 * NLSE conserves; a state whose output mass is 0 is left as it is.  psi_out
 * must not overlap psi_in. */
int nlse_sur_forward(nlse_sur_t s, int nb, const void *psi_in, void *psi_out, int project_mass, double *masses_out);

/* Weight of the mass term of the training loss (see above), >= 0. */
int nlse_sur_set_mass_weight(nlse_sur_t s, double mass_weight);

/* Relative L2 distance ||a_b - b_b|| / ||b_b|| of nb state pairs (device
 * float2 [nb][H][W] each) in FP64 with a fixed summation order, into the
 * host array rel_l2_host[nb]; synchronises the stream.  (The rollout's check
 * of a predicted window against the RK4 window.) */
int nlse_sur_compare(nlse_sur_t s, int nb, const void *a, const void *b, double *rel_l2_host);

/* Loss gradient w.r.t. every parameter for (psi_in, psi_target) into grad_out
 * (device, param layout; NULL to skip) and the loss into *loss_out (host;
 * NULL to skip, else synchronises). */
int nlse_sur_gradients(nlse_sur_t s, int nb, const void *psi_in, const void *psi_target, float *grad_out,
                       double *loss_out);

/* One Adam step on a batch (forward, backward, update); *loss_out as above.
 * noise > 0 trains on psi_in + noise * max|psi_in| * (g + i g'), g and g'
 * standard normal per site (drawn in the kernel from a counter-based
 * SplitMix64 stream seeded by nlse_sur_init's seed and the step count), with
 * the residual taken from that noisy input: the network learns to map
 * slightly perturbed states, like its own predictions, onto the clean next
 * window.  NLSE_EINVAL for lr <= 0 or noise < 0. */
int nlse_sur_train_step(nlse_sur_t s, int nb, const void *psi_in, const void *psi_target, float lr, float noise,
                        double *loss_out);

/* Convolution kernels: 1 (default) runs the forward and backward-data
 * convolutions of layers whose gathered and output channel counts are
 * multiples of 16 (output channels 16..256, dilation <= 16) on the tcgen05
 * tensor-core kernel (TMEM accumulators); 0 keeps every convolution on the
 * mma.sync kernels.  Both give the same results up to FP32 summation order.
 * NLSE_EINVAL for other values. */
int nlse_sur_set_kernel(nlse_sur_t s, int tensor_core_gen);

/* Wait for the stream.  NLSE_ETIMEOUT if a bounded wait inside a tcgen05
 * kernel ran out since the last check (the kernel then stopped early and its
 * outputs are incomplete); gradients / train_step report the same when they
 * return a loss. */
int nlse_sur_sync(nlse_sur_t s);

int nlse_sur_destroy(nlse_sur_t s);

/*
 * Mass h^d sum |Psi|^2 for callers that cannot allocate device memory.
 * The paper has no counterpart; it exists for code that may not call
 * cudaMalloc: work issued while another component captures the stream into
 * a CUDA graph (allocation is illegal there), plug-ins whose host
 * application owns all device memory through its own pool, and real-time
 * loops that cannot take the device synchronisation an allocation may
 * imply.  Such callers cannot create a context (it needs a workspace).
 *   dims, N, h  the grid as in nlse_create (any N[k] >= 1)
 *   dtype       NLSE_C128 / NLSE_C64_ACC64 (psi is double2) or NLSE_C64 (float2)
 *   psi         device input;  out: device pointer to one double (the result)
 *   stream      cudaStream_t as void* (NULL = legacy default stream)
 * Asynchronous; the result is in *out once the stream reaches it.  The
 * reduction's scratch (one pair of FP64 partial sums per block of 4096
 * sites) is a fixed 128 KiB array inside the library that every GPU which
 * loads the library keeps until the process exits, so grids above
 * 8192 * 4096 = 33,554,432 sites are rejected with NLSE_EINVAL.  Nothing is
 * allocated and no allocating library routine is called.  The first call on
 * a device (with that device current) looks up the array's device address
 * once; make that first call before any stream capture.  All calls share the
 * array: calls whose kernels overlap on the GPU (several streams or host
 * threads at once) race and must be serialised by the caller.  A NaN or Inf
 * in psi yields a non-finite result (no status flag).  Errors: NLSE_EINVAL,
 * NLSE_ECUDA, with the message in nlse_last_error().
 */
int nlse_mass_noalloc(int dims, const int64_t *N, double h, int dtype, const void *psi, double *out,
                      void *stream);

/*
 * Test hooks (not needed in normal use).
 *   NLSE_DEBUG_SPIN_LIMIT  value = SM clock cycles any device-side wait may
 *                          last before the kernel gives up (default ~2e9,
 *                          about a second).
 *   NLSE_DEBUG_EXTRA_TX    value = extra bytes (multiple of 16, <= 2^20) that
 *                          every TMA barrier of the 3D tiled kernel expects
 *                          beyond what its copy delivers, so its wait runs out
 *                          without any fault; the next nlse_sync then returns
 *                          NLSE_ETIMEOUT once.  0 restores normal operation.
 *   NLSE_DEBUG_FIX_OFFSET  value (-64..64) added to the exact-sum stencil's
 *                          fraction bits after they are derived from Psi:
 *                          positive values shrink its range below the state,
 *                          so that the FP64 out-of-range fallback runs at
 *                          every site; 0 restores normal operation.
 * Psi is not valid after a step that timed out; reporting NLSE_ETIMEOUT
 * clears every status flag (including a non-finite flag the invalid step
 * may have raised), and the context stays usable once Psi is restored.
 */
#define NLSE_DEBUG_SPIN_LIMIT 1
#define NLSE_DEBUG_EXTRA_TX   2
#define NLSE_DEBUG_FIX_OFFSET 3
int nlse_debug_set(nlse_t ctx, int key, long long value);

#ifdef __cplusplus
}
#endif
#endif /* NLSE_H */
