// The C ABI of include/nlse.h: argument checks, workspace layout, stage
// dispatch, CUDA-graph chunking of the step loop, reductions and errors.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>

#include "../../include/nlse.h"
#include "nlse_internal.h"

using namespace nlse;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(NLSE_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

constexpr int kGraphSteps = 16;   // RK4 steps captured per graph replay
constexpr long long kSpinLimit = 2000000000ll;   // ~1 s of SM clock: bound on device-side waits
constexpr unsigned int kFlagTimeoutBit = 4u;

// cuTensorMapEncodeTiled, resolved once through the runtime (no link to libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t ktot, ptmp, pout, pn32, vs, alt, partials, status, total;
};

bool layout_for(int dims, const int64_t* N, int dtype, Layout* L, int64_t* total_sites) {
  if (dims < 1 || dims > 3 || !N) return false;
  if (dtype < NLSE_C128 || dtype > NLSE_C64_ACC64) return false;
  int64_t total = 1;
  for (int k = 0; k < dims; ++k) {
    if (N[k] < 3 || N[k] > (int64_t(1) << 30)) return false;
    total *= N[k];
    if (total > (int64_t(1) << 40)) return false;
  }
  const size_t es = (dtype == NLSE_C128) ? 16 : 8;
  size_t off = 0;
  L->ktot = off; off = align_up(off + es * total);
  L->ptmp = off; off = align_up(off + es * total);
  L->pout = off; off = align_up(off + es * total);
  L->pn32 = off; if (dtype == NLSE_C64_ACC64) off = align_up(off + 8 * total);
  L->vs = off; if (dtype == NLSE_C128) off = align_up(off + 8 * total);   // V / cLF for the exact-sum stages
  L->alt = off; if (dtype == NLSE_C64 && dims == 3) off = align_up(off + 8 * total);   // Psi ping-pong (fused step)
  L->partials = off; off = align_up(off + sizeof(double) * 2 * kMaxReduceBlocks);
  L->status = off; off = align_up(off + 256);
  L->total = off;
  if (total_sites) *total_sites = total;
  return true;
}

}  // namespace

struct nlse_ctx {
  int d;
  int64_t n[3];
  int64_t total;
  double h, a, s;
  int bc, order, dtype;
  void* psi;
  const void* V;
  cudaStream_t stream;
  char* ws;
  Layout lay;
  double vmax;
  int fixF;          // reference fraction bits F0 of the exact-sum stencil (FP64 path): cLF = cL 2^-F0
  int fix_offset;    // test hook added to the derived fraction bits (nlse_debug_set)
  int variant, tile_cfg;
  cudaStream_t cap;
  cudaGraphExec_t exec;
  double graph_dt;
  int graph_variant;
  // TMA descriptors of the stage inputs (Psi or its FP32 copy, Psi_tmp, Psi_out) per tile shape
  CUtensorMap tmaps[4][3];
  signed char tmap_state[4][3];   // 0 = not built, 1 = ok, -1 = layout not eligible
  CUtensorMap fmaps[3];           // the fused kernel's inputs: Psi, its ping-pong copy, Psi_out
  signed char fmap_state[3];
  long long spin_limit;           // bound on device-side waits (cycles)
  unsigned int extra_tx;          // test hook, see nlse_debug_set
  bool line_failed;               // the 1D cluster path could not be launched here: per-site kernel instead
  cudaStream_t side;              // wall-shell kernels run here, concurrently with the deep kernels
  cudaEvent_t ev_fork, ev_join;
  cudaStream_t side_yx[2];        // 3D: the y- and x-wall slabs' streams
  cudaEvent_t ev_join_yx[2];

  void* at(size_t off) const { return ws + off; }
  unsigned int* flag() const { return (unsigned int*)(ws + lay.status); }
  unsigned long long* vbits() const { return (unsigned long long*)(ws + lay.status + 8); }
  int* fdev() const { return (int*)(ws + lay.status + 16); }                    // current fraction bits
  unsigned int* emax() const { return (unsigned int*)(ws + lay.status + 20); }  // stage-4 largest exponent
  bool exact() const { return dtype == NLSE_C128 && variant >= 2 && variant <= 3; }
  double* result() const { return (double*)(ws + lay.status + 64); }
  double* partials() const { return (double*)(ws + lay.partials); }
};

namespace {

// Tile shape in use: the caller's choice, else the measured default per form
// and size (nlse_autotune can refine it): 32x8 for FP64; for the FP32 forms
// in 3D, 64x8 on planes of at least 8192 sites (fewer, wider TMA boxes; 100^3:
// 65.7 against 68.5 us per step, 128^3: 88.3 against 92.1) and 32x8 on smaller
// planes (enough CTAs to fill the SMs; 64^3: 41.8 against 43.3); 32x16 in 2D.
int resolved_tile(const nlse_ctx* c) {
  if (c->tile_cfg >= 0) return c->tile_cfg;
  if (c->dtype == NLSE_C128) return 0;
  if (c->d == 3) return c->n[1] * c->n[2] >= 8192 ? 3 : 0;
  return 2;
}

template <class T>
Field<T> make_field(const nlse_ctx* c, const void* in) {
  using R = typename T::R;
  Field<T> f;
  memset(&f, 0, sizeof(f));
  for (int k = 0; k < 3; ++k) { f.n[k] = 1; f.m[k] = 1; f.st[k] = 0; }
  int64_t stride = 1;
  for (int k = c->d - 1; k >= 0; --k) {
    f.n[k] = int(c->n[k]);
    f.m[k] = int(c->n[k] - 2);
    f.st[k] = stride;
    stride *= c->n[k];
  }
  f.ninterior = 1;
  for (int k = 0; k < c->d; ++k) f.ninterior *= (c->n[k] - 2);
  f.a = R(c->a);
  f.s = R(c->s);
  f.h2_over_a = R(c->h * c->h / c->a);
  f.cL = R(c->order == 4 ? c->a / (12.0 * c->h * c->h) : c->a / (c->h * c->h));
  f.tiny = R(sizeof(R) == 8 ? 1e-300 : 1e-30);
  f.bc = c->bc;
  f.F = c->fixF;
  f.Fdev = (c->dtype == NLSE_C128) ? c->fdev() : nullptr;
  f.cLF = ldexp(c->order == 4 ? c->a / (12.0 * c->h * c->h) : c->a / (c->h * c->h), -c->fixF);
  f.invcLF = R(1.0 / f.cLF);
  f.sG = R(c->s / f.cLF);
  f.V = (const typename T::VR*)c->V;
  f.in = (const typename T::C*)in;
  return f;
}

LaunchCfg launch_cfg(const nlse_ctx* c);

template <class T>
cudaError_t dispatch_stage(const nlse_ctx* c, const StageArgs<T>& A, const void* tmap, cudaStream_t st) {
  LaunchCfg L = launch_cfg(c);
  L.variant = (c->variant == 4) ? 1 : c->variant;   // single stages of the fused variant: the tiled kernel
  L.tmap = tmap;
  switch (c->d * 10 + c->order) {
    case 12: return launch_stage<T, 1, 2>(A, L, st);
    case 14: return launch_stage<T, 1, 4>(A, L, st);
    case 22: return launch_stage<T, 2, 2>(A, L, st);
    case 24: return launch_stage<T, 2, 4>(A, L, st);
    case 32: return launch_stage<T, 3, 2>(A, L, st);
    default: return launch_stage<T, 3, 4>(A, L, st);
  }
}

// A 3D TMA descriptor over a complex field of the context's shape (real components of es bytes) with a
// box of box_x components by box_y rows by one plane; false when the layout is not eligible (TMA needs
// 16-byte row pitches and a 16-byte aligned base).
bool encode_field_map(const nlse_ctx* c, CUtensorMap* m, const void* ptr, size_t es, int box_x, int box_y) {
  const cuuint64_t nx = c->n[2], ny = c->n[1], nz = c->n[0];
  EncodeTiledFn fn = encode_fn();
  if (!fn || (2 * nx * es) % 16 != 0 || ((uintptr_t)ptr % 16) != 0) return false;
  cuuint64_t dims[3] = {2 * nx, ny, nz};
  cuuint64_t strides[2] = {2 * nx * es, 2 * nx * ny * es};
  cuuint32_t box[3] = {cuuint32_t(box_x), cuuint32_t(box_y), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(ptr),
            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The fused kernel's TMA descriptor of buffer `buf` (0 = Psi, 1 = its ping-pong copy, 2 = Psi_out).
const CUtensorMap* fused_tmap(const nlse_ctx* cc, int buf, const void* ptr) {
  nlse_ctx* c = const_cast<nlse_ctx*>(cc);
  signed char& st = c->fmap_state[buf];
  if (st == 0) st = encode_field_map(c, &c->fmaps[buf], ptr, 4, kFusedBoxX, kFusedBoxY) ? 1 : -1;
  return st == 1 ? &c->fmaps[buf] : nullptr;
}

// The fused step runs for the FP32 form on 3D grids with every extent >= 16
// and TMA-eligible rows, except on periodic grids (their shell wraps).
bool fused_path(const nlse_ctx* c) {
  if (c->variant != 4 || c->dtype != NLSE_C64 || c->d != 3 || c->bc == NLSE_BC_PERIODIC) return false;
  const int n[3] = {int(c->n[0]), int(c->n[1]), int(c->n[2])};
  if (!fused_grid_ok(3, n)) return false;
  return fused_tmap(c, 0, c->psi) && fused_tmap(c, 1, c->at(c->lay.alt)) && fused_tmap(c, 2, c->at(c->lay.pout));
}

// The TMA descriptor of stage-input buffer `buf` (0 = Psi or its FP32 copy,
// 1 = Psi_tmp, 2 = Psi_out) for the 3D tiled kernel's tile, or nullptr when
// the layout is not eligible (TMA needs 16-byte row pitches).
const CUtensorMap* stage_tmap(const nlse_ctx* cc, int buf, const void* ptr) {
  nlse_ctx* c = const_cast<nlse_ctx*>(cc);
  if (c->d != 3 || (c->variant != 1 && c->variant != 2 && c->variant != 4)) return nullptr;
  const int tc = resolved_tile(c);
  signed char& st = c->tmap_state[tc][buf];
  if (st == 0) {
    st = -1;
    int tx, ty;
    tma_tile_shape(tc, &tx, &ty);
    const size_t es = (c->dtype == NLSE_C128) ? 8 : 4;   // bytes of one real component
    const cuuint64_t nx = c->n[2], ny = c->n[1], nz = c->n[0];
    EncodeTiledFn fn = encode_fn();
    if (fn && (2 * nx * es) % 16 == 0 && ((uintptr_t)ptr % 16) == 0) {
      cuuint64_t dims[3] = {2 * nx, ny, nz};
      cuuint64_t strides[2] = {2 * nx * es, 2 * nx * ny * es};
      cuuint32_t box[3] = {cuuint32_t(2 * (tx + 4)), cuuint32_t(ty + 4), 1};
      cuuint32_t estr[3] = {1, 1, 1};
      CUresult r = fn(&c->tmaps[tc][buf], es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                      const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r == CUDA_SUCCESS) st = 1;
    }
  }
  return st == 1 ? &c->tmaps[tc][buf] : nullptr;
}

// The arguments of stage s (1..4) of Eq. RK4_GPU: Psi -> Psi_tmp -> Psi_out ->
// Psi_tmp -> Psi.  cur holds Psi^n, stage 4 writes Psi^{n+1} to nxt (the same
// buffer except on the fused path's ping-pong steps).
template <class T>
StageArgs<T> stage_args(const nlse_ctx* c, int s, double dt, void* cur, void* nxt) {
  using C = typename T::C;
  using R = typename T::R;
  const bool mix = (c->dtype == NLSE_C64_ACC64);
  C* ktot = (C*)c->at(c->lay.ktot);
  C* ptmp = (C*)c->at(c->lay.ptmp);
  C* pout = (C*)c->at(c->lay.pout);
  const C* psin = mix ? (const C*)c->at(c->lay.pn32) : (const C*)cur;
  const void* in[4] = {psin, ptmp, pout, ptmp};
  C* outs[4] = {ptmp, pout, ptmp, nullptr};
  const double dtc[4] = {dt / 2.0, dt / 2.0, dt, dt / 6.0};
  const int i = s - 1;
  StageArgs<T> A;
  memset(&A, 0, sizeof(A));
  A.f = make_field<T>(c, in[i]);
  A.psin = psin;
  A.ktot = ktot;
  A.out = outs[i];
  A.master = (typename T::M*)nxt;
  A.master_in = (const typename T::M*)cur;
  A.n32 = mix ? (C*)c->at(c->lay.pn32) : nullptr;
  // FP64 with the exact-sum stencil: F is formed in units of cLF, so the stage coefficient carries it
  const bool g = std::is_same<T, P64>::value && c->exact();
  A.dtc = R(g ? dtc[i] * A.f.cLF : dtc[i]);
  A.dt6 = dt / 6.0;
  A.stage = s;
  A.flag = c->flag();
  A.Vs = (g && c->V) ? (const typename T::VR*)c->at(c->lay.vs) : nullptr;
  A.emax = (g && s == 4) ? c->emax() : nullptr;   // collects the exponent of Psi^{n+1}
  return A;
}

// Stage s of one step, Psi updated in place.
template <class T>
cudaError_t launch_one_stage(const nlse_ctx* c, int s, double dt, cudaStream_t st) {
  const StageArgs<T> A = stage_args<T>(c, s, dt, c->psi, c->psi);
  const int inbuf[4] = {0, 1, 2, 1};
  return dispatch_stage<T>(c, A, stage_tmap(c, inbuf[s - 1], A.f.in), st);
}

LaunchCfg launch_cfg(const nlse_ctx* c) {
  LaunchCfg L;
  L.variant = c->variant;
  L.tile_cfg = resolved_tile(c);
  L.tmap = nullptr;
  L.spin_limit = c->spin_limit;
  L.extra_tx = c->extra_tx;
  L.side = c->side;
  L.ev_fork = c->ev_fork;
  L.ev_join = c->ev_join;
  for (int i = 0; i < 2; ++i) {
    L.side_yx[i] = c->side_yx[i];
    L.ev_join_yx[i] = c->ev_join_yx[i];
  }
  return L;
}

// 1D lines that take the cluster path: FP64 or FP32 (not the mixed form), variant 1, 2 or 4.
bool line_path(const nlse_ctx* c) {
  if (c->d != 1 || c->line_failed || c->dtype == NLSE_C64_ACC64) return false;
  if (c->variant != 1 && c->variant != 2 && c->variant != 4) return false;
  return line_ok(int(c->n[0]), c->dtype == NLSE_C128);
}

cudaError_t launch_line(const nlse_ctx* c, int64_t nsteps, double dt) {
  if (c->dtype == NLSE_C128) {
    StageArgs<P64> A[4];
    for (int s = 1; s <= 4; ++s) A[s - 1] = stage_args<P64>(c, s, dt, c->psi, c->psi);
    return launch_line_steps<P64>(A, nsteps, int(c->n[0]), c->order, c->exact(), c->fixF, c->fix_offset, c->stream);
  }
  StageArgs<P32> A[4];
  for (int s = 1; s <= 4; ++s) A[s - 1] = stage_args<P32>(c, s, dt, c->psi, c->psi);
  return launch_line_steps<P32>(A, nsteps, int(c->n[0]), c->order, false, c->fixF, c->fix_offset, c->stream);
}

// One step of the fused path from buffer cur to buffer nxt (Psi or its ping-pong copy).
cudaError_t launch_step_fused(const nlse_ctx* c, double dt, cudaStream_t st, void* cur, void* nxt) {
  StageArgs<P32> A[4];
  for (int s = 1; s <= 4; ++s) A[s - 1] = stage_args<P32>(c, s, dt, cur, nxt);
  const CUtensorMap* tm12 = fused_tmap(c, cur == c->psi ? 0 : 1, cur);
  const CUtensorMap* tm34 = fused_tmap(c, 2, c->at(c->lay.pout));
  const LaunchCfg L = launch_cfg(c);
  return c->order == 4 ? launch_fused_step<4>(A, tm12, tm34, L, st) : launch_fused_step<2>(A, tm12, tm34, L, st);
}

// The exact-sum stencil's scale for the next step: from the exponent stage 4
// collected (psi == nullptr) or from a full pass over psi.
cudaError_t update_fix(const nlse_ctx* c, const void* psi, cudaStream_t st) {
  return launch_fix_update((const double*)psi, 2 * c->total, c->emax(), c->fdev(), c->fixF, c->fix_offset, st);
}

template <class T>
cudaError_t launch_step(const nlse_ctx* c, double dt, cudaStream_t st) {
  for (int s = 1; s <= 4; ++s) {
    cudaError_t e = launch_one_stage<T>(c, s, dt, st);
    if (e != cudaSuccess) return e;
  }
  if (std::is_same<T, P64>::value && c->exact()) return update_fix(c, nullptr, st);
  return cudaSuccess;
}

cudaError_t launch_stage_any(const nlse_ctx* c, int s, double dt, cudaStream_t st) {
  switch (c->dtype) {
    case NLSE_C128: return launch_one_stage<P64>(c, s, dt, st);
    case NLSE_C64: return launch_one_stage<P32>(c, s, dt, st);
    default: return launch_one_stage<PMix>(c, s, dt, st);
  }
}

cudaError_t launch_step_any(const nlse_ctx* c, double dt, cudaStream_t st) {
  switch (c->dtype) {
    case NLSE_C128: return launch_step<P64>(c, dt, st);
    case NLSE_C64: return launch_step<P32>(c, dt, st);
    default: return launch_step<PMix>(c, dt, st);
  }
}

void drop_graph(nlse_ctx* c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  c->exec = nullptr;
}

int ensure_graph(nlse_ctx* c, double dt) {
  if (c->exec && c->graph_dt == dt) return NLSE_OK;
  drop_graph(c);
  if (!c->cap) {
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  }
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
  cudaError_t le = cudaSuccess;
  const bool fused = fused_path(c);
  for (int i = 0; i < kGraphSteps && le == cudaSuccess; ++i) {
    if (fused) {   // ping-pong: even steps Psi -> copy, odd steps copy -> Psi (kGraphSteps is even)
      void* a = c->psi;
      void* b = c->at(c->lay.alt);
      le = (i % 2 == 0) ? launch_step_fused(c, dt, c->cap, a, b) : launch_step_fused(c, dt, c->cap, b, a);
    } else {
      le = launch_step_any(c, dt, c->cap);
    }
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->cap, &g);
  if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(le, "stage launch (capture)"); }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&c->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { c->exec = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
  c->graph_dt = dt;
  c->graph_variant = c->variant;
  return NLSE_OK;
}

__global__ void k_round_master(const double2* __restrict__ m, float2* __restrict__ o, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = m[i];
    o[i] = make_float2(float(v.x), float(v.y));
  }
}

int read_status(nlse_ctx* c) {
  unsigned int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, c->flag(), sizeof(flag), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (flag & kFlagTimeoutBit) {
    // Report once and clear every status bit: nothing a timed-out step wrote
    // is valid (a non-finite value it produced included); the caller restores
    // Psi and the context stays usable.
    const unsigned int keep = 0;
    cudaMemcpyAsync(c->flag(), &keep, sizeof(keep), cudaMemcpyHostToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
    return fail(NLSE_ETIMEOUT, "a bounded device-side wait gave up (a TMA copy did not complete)");
  }
  if (flag & 3u) return fail(NLSE_ENONFINITE, "non-finite value in Psi");
  return NLSE_OK;
}

}  // namespace

namespace nlse {
// Lets other translation units of the library report through nlse_last_error().
void record_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

// cuTensorMapEncodeTiled for other translation units (nullptr when unavailable).
void* tensor_map_encoder() { return reinterpret_cast<void*>(encode_fn()); }

__global__ void k_scale_v(const double* __restrict__ V, double s, int64_t n, double* __restrict__ Vs) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Vs[i] = V[i] * s;
}

cudaError_t launch_scale_v(const double* V, double s, int64_t n, double* Vs, cudaStream_t stream) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  k_scale_v<<<(unsigned)b, 256, 0, stream>>>(V, s, n, Vs);
  return cudaGetLastError();
}

cudaError_t launch_round_master(const double2* master, float2* n32, int64_t total, cudaStream_t stream) {
  int64_t b = (total + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  k_round_master<<<(unsigned)b, 256, 0, stream>>>(master, n32, total);
  return cudaGetLastError();
}
}  // namespace nlse

extern "C" {

const char* nlse_last_error(void) { return g_err; }

size_t nlse_workspace_bytes(int dims, const int64_t* N, int dtype) {
  Layout L;
  if (!layout_for(dims, N, dtype, &L, nullptr)) return 0;
  return L.total;
}

double nlse_max_dt(int dims, double h, double a, int order, double vmax, double s_rho_max) {
  if (dims < 1 || dims > 3 || !(h > 0) || !(a > 0) || (order != 2 && order != 4)) return -1.0;
  // spectral radius of Lap on the grid: 4d/h^2 (CD), 16d/(3h^2) (2SHOC); RK4 reaches 2 sqrt(2) on i R
  const double rho = (order == 4 ? 16.0 * dims / 3.0 : 4.0 * dims) / (h * h);
  return 2.0 * sqrt(2.0) / (a * rho + fabs(vmax) + fabs(s_rho_max));
}

int nlse_create(nlse_t* out, int dims, const int64_t* N, double h, double a, double s, const void* V, int bc,
                int order, int dtype, void* psi, void* workspace, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  if (!out) return fail(NLSE_EINVAL, "out is NULL");
  *out = nullptr;
  Layout L;
  int64_t total = 0;
  if (!layout_for(dims, N, dtype, &L, &total))
    return fail(NLSE_EINVAL, "bad dims/N/dtype (dims in 1..3, every N >= 3, dtype 0..2)");
  if (!(h > 0) || !isfinite(h)) return fail(NLSE_EINVAL, "h must be > 0");
  if (!(a > 0) || !isfinite(a)) return fail(NLSE_EINVAL, "a must be > 0");
  if (!isfinite(s)) return fail(NLSE_EINVAL, "s must be finite");
  if (bc != NLSE_BC_DIRICHLET && bc != NLSE_BC_MSD && bc != NLSE_BC_L0 && bc != NLSE_BC_PERIODIC)
    return fail(NLSE_EINVAL, "bc must be 0, 1, 2 or 3");
  if (order != 2 && order != 4) return fail(NLSE_EINVAL, "order must be 2 or 4");
  if (!psi) return fail(NLSE_EINVAL, "psi is NULL");
  if (!workspace) return fail(NLSE_EINVAL, "workspace is NULL");
  if ((uintptr_t)workspace % kAlign) return fail(NLSE_EINVAL, "workspace must be 256-byte aligned");
  if ((uintptr_t)psi % 16 || (V && (uintptr_t)V % 8)) return fail(NLSE_EINVAL, "psi/V misaligned");
  if (ws_bytes < L.total) return fail(NLSE_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, L.total);

  nlse_ctx* c = new nlse_ctx();
  memset(c, 0, sizeof(*c));
  c->d = dims;
  for (int k = 0; k < 3; ++k) c->n[k] = (k < dims) ? N[k] : 1;
  c->total = total;
  c->h = h; c->a = a; c->s = s;
  c->bc = bc; c->order = order; c->dtype = dtype;
  c->psi = psi; c->V = V;
  c->stream = (cudaStream_t)stream;
  c->ws = (char*)workspace;
  c->lay = L;
  // Default kernel per form and size, from timings of the paper's workloads (MSD, 2SHOC, us per step):
  // FP64 takes the exact-sum stencil on the tiled kernels, except where the grid is so small that a
  // step is bound by latency, not by the FP64 pipe's throughput, and the plain FP64 stencil's shorter
  // instruction chain wins: 3D grids of at most 2^15 sites (one thread per site; 21^3: 62.6 against
  // 93.7 for the tiled exact-sum kernel, 32^3: 67.2 against 95.9; 36^3: 89.7 against 86.3), 2D grids of
  // at most 80,000 sites (tiled; 100^2: 32.9 against 51.7, 282^2: 49.7 against 56.6; 316^2: 61.1
  // against 54.0) and 1D lines: up to 2500 sites on the cluster path (2001 sites: 14.3 against 19.7
  // with the exact-sum stencil, 18.1 against 19.4 for one thread per site on the dark soliton), up to
  // 2^15 sites one thread per site (beyond ~2500 sites the cluster's 16 SMs bound it: 10,000 sites 34.8
  // against 19.0; 20,000: 21.5 against 23.8 with the exact-sum stencil; 100,000: 36.9 against 29.0).
  // The FP32 forms take the tiled kernel on 3D grids above 2^17 sites (64^3: 41.8 against 47.1 for one
  // thread per site, 128^3: 88.3 against 176.8; 46^3: 39.2 against 34.5).
  c->variant = (dtype == NLSE_C128) ? 2 : 1;
  if (dims == 3 && total <= (dtype == NLSE_C128 ? (int64_t(1) << 15) : (int64_t(1) << 17))) c->variant = 0;
  if (dims == 2 && dtype == NLSE_C128 && total <= 80000) c->variant = 1;
  if (dims == 1 && dtype == NLSE_C128)
    c->variant = (total <= 2500 && line_ok(int(N[0]), true)) ? 1 : (total <= (int64_t(1) << 15) ? 0 : 3);
  c->tile_cfg = -1;
  c->spin_limit = kSpinLimit;
  c->graph_dt = -1.0;

  cudaError_t e = cudaMemsetAsync(c->at(L.status), 0, 256, c->stream);
  if (e == cudaSuccess && V) {
    e = launch_vmax(V, dtype == NLSE_C128, total, c->vbits(), c->stream);
    unsigned long long bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, c->vbits(), sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    memcpy(&c->vmax, &bits, sizeof(double));
  }
  if (e == cudaSuccess && dims >= 2) {
    e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess && dims == 3; ++i) {
      e = cudaStreamCreateWithFlags(&c->side_yx[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join_yx[i], cudaEventDisableTiming);
    }
  }
  // Exact-sum stencil reference scale F0: the largest component of Psi0 below
  // 2^53 in fixed point (operands are accepted below 2^55).
  c->fixF = 52;
  if (e == cudaSuccess && dtype == NLSE_C128) {
    e = launch_vmax(psi, true, 2 * total, c->vbits(), c->stream);
    unsigned long long bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, c->vbits(), sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    double pmax = 0.0;
    memcpy(&pmax, &bits, sizeof(double));
    if (pmax > 0.0 && isfinite(pmax)) {
      int ex = 0;
      frexp(pmax, &ex);              // pmax < 2^ex
      c->fixF = 56 - (ex + 3);
    }
  }
  if (e == cudaSuccess && dtype == NLSE_C128 && V) {   // V / cLF for the exact-sum stages
    const Field<P64> f = make_field<P64>(c, psi);
    e = launch_scale_v((const double*)V, 1.0 / f.cLF, total, (double*)c->at(L.vs), c->stream);
  }
  if (e == cudaSuccess && dtype == NLSE_C128) e = update_fix(c, psi, c->stream);
  if (e != cudaSuccess) {
    nlse_destroy(c);
    return cuda_fail(e, "nlse_create");
  }
  *out = c;
  return NLSE_OK;
}

int nlse_set_kernel(nlse_t c, int variant, int tile_cfg) {
  if (!c) return fail(NLSE_EINVAL, "NULL context");
  if (variant < 0 || variant > 4) return fail(NLSE_EINVAL, "variant must be 0..4");
  if (tile_cfg < -1 || tile_cfg > 3) return fail(NLSE_EINVAL, "tile_cfg must be -1..3");
  c->variant = variant;
  c->tile_cfg = tile_cfg;
  drop_graph(c);
  return NLSE_OK;
}

int nlse_kernel_in_use(nlse_t c) {
  if (!c) return fail(NLSE_EINVAL, "NULL context");
  if (fused_path(c)) return 4;
  if (line_path(c)) return c->exact() ? 2 : 1;
  if (c->variant == 4) return c->d == 1 ? 0 : 1;
  if (c->d == 1) return (c->dtype == NLSE_C128 && c->variant >= 2) ? 3 : 0;
  if (c->dtype != NLSE_C128 && c->variant >= 2) return c->variant - 2;
  return c->variant;
}

int nlse_refresh_potential(nlse_t c) {
  if (!c) return fail(NLSE_EINVAL, "NULL context");
  cudaError_t e = cudaSuccess;
  double vmax = 0.0;
  if (c->V) {
    e = launch_vmax(c->V, c->dtype == NLSE_C128, c->total, c->vbits(), c->stream);
    unsigned long long bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, c->vbits(), sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    memcpy(&vmax, &bits, sizeof(double));
    if (e == cudaSuccess && c->dtype == NLSE_C128) {
      const Field<P64> f = make_field<P64>(c, c->psi);
      e = launch_scale_v((const double*)c->V, 1.0 / f.cLF, c->total, (double*)c->at(c->lay.vs), c->stream);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "nlse_refresh_potential");
  c->vmax = vmax;
  return NLSE_OK;
}

int nlse_step(nlse_t c, int64_t nsteps, double dt) {
  if (!c) return fail(NLSE_EINVAL, "NULL context");
  if (nsteps < 0) return fail(NLSE_EINVAL, "nsteps < 0");
  if (!(dt > 0) || !isfinite(dt)) return fail(NLSE_EINVAL, "dt must be > 0");
  const double bound = nlse_max_dt(c->d, c->h, c->a, c->order, c->vmax, 0.0);
  if (dt > bound) return fail(NLSE_EUNSTABLE, "dt = %g above the RK4 linear stability bound %g", dt, bound);
  if (nsteps == 0) return NLSE_OK;
  cudaError_t e = cudaSuccess;
  if (c->dtype == NLSE_C64_ACC64)
    e = launch_round_master((const double2*)c->psi, (float2*)c->at(c->lay.pn32), c->total, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "round master");
  // the exact-sum scale of the state as the caller left it (stage 4 keeps it current from here on)
  if (c->exact() && (e = update_fix(c, c->psi, c->stream)) != cudaSuccess) return cuda_fail(e, "scale");
  if (line_path(c)) {   // 1D: the whole call on one thread-block cluster
    e = launch_line(c, nsteps, dt);
    if (e == cudaSuccess) return NLSE_OK;
    if (e != cudaErrorInvalidConfiguration) return cuda_fail(e, "line launch");
    cudaGetLastError();
    c->line_failed = true;   // cannot be co-scheduled here: the per-site kernel from now on
  }
  int64_t left = nsteps;
  if (nsteps >= kGraphSteps) {
    int rc = ensure_graph(c, dt);
    if (rc != NLSE_OK) return rc;
    for (; left >= kGraphSteps; left -= kGraphSteps) {
      e = cudaGraphLaunch(c->exec, c->stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    }
  }
  for (; left > 0; --left) {
    e = launch_step_any(c, dt, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stage launch");
  }
  return NLSE_OK;
}

int nlse_rhs(nlse_t c, const void* psi_in, void* F_out) {
  if (!c || !psi_in || !F_out) return fail(NLSE_EINVAL, "NULL argument");
  cudaError_t e;
  if (c->exact() && (e = update_fix(c, psi_in, c->stream)) != cudaSuccess) return cuda_fail(e, "scale");
  auto run = [&](auto tag) {
    using T = decltype(tag);
    StageArgs<T> A;
    memset(&A, 0, sizeof(A));
    A.f = make_field<T>(c, psi_in);
    A.out = (typename T::C*)F_out;
    A.stage = 0;
    A.flag = c->flag();
    const bool g = std::is_same<T, P64>::value && c->variant >= 2;   // F in units of cLF: scale it back
    A.dtc = typename T::R(g ? A.f.cLF : 1.0);
    A.Vs = (g && c->V) ? (const typename T::VR*)c->at(c->lay.vs) : nullptr;
    return dispatch_stage<T>(c, A, nullptr, c->stream);
  };
  if (c->dtype == NLSE_C128) e = run(P64{});
  else if (c->dtype == NLSE_C64) e = run(P32{});
  else e = run(PMix{});
  if (e != cudaSuccess) return cuda_fail(e, "rhs launch");
  return NLSE_OK;
}

int nlse_mass(nlse_t c, double* out_host) {
  if (!c || !out_host) return fail(NLSE_EINVAL, "NULL argument");
  cudaError_t e = launch_mass(c->psi, c->dtype != NLSE_C64, c->total, pow(c->h, c->d), c->partials(), c->result(),
                              c->flag(), c->stream);
  double v = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, c->result(), sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mass");
  int rc = read_status(c);
  if (rc != NLSE_OK) return rc;
  *out_host = v;
  return NLSE_OK;
}

int nlse_energy(nlse_t c, double* out_host) {
  if (!c || !out_host) return fail(NLSE_EINVAL, "NULL argument");
  const double scale = pow(c->h, c->d);
  cudaError_t e;
  auto run = [&](auto tag) {
    using T = decltype(tag);
    Field<T> f = make_field<T>(c, c->psi);
    switch (c->d * 10 + c->order) {
      case 12: return launch_energy<T, 1, 2>(f, scale, c->partials(), c->result(), c->flag(), c->stream);
      case 14: return launch_energy<T, 1, 4>(f, scale, c->partials(), c->result(), c->flag(), c->stream);
      case 22: return launch_energy<T, 2, 2>(f, scale, c->partials(), c->result(), c->flag(), c->stream);
      case 24: return launch_energy<T, 2, 4>(f, scale, c->partials(), c->result(), c->flag(), c->stream);
      case 32: return launch_energy<T, 3, 2>(f, scale, c->partials(), c->result(), c->flag(), c->stream);
      default: return launch_energy<T, 3, 4>(f, scale, c->partials(), c->result(), c->flag(), c->stream);
    }
  };
  if (c->dtype == NLSE_C128) e = run(P64{});
  else if (c->dtype == NLSE_C64) e = run(E32{});
  else e = run(EMix{});
  double v = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, c->result(), sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "energy");
  int rc = read_status(c);
  if (rc != NLSE_OK) return rc;
  *out_host = v;
  return NLSE_OK;
}

namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;   // process-wide cache: context key -> tile_cfg

std::string tune_key(const nlse_ctx* c) {
  char b[160];
  snprintf(b, sizeof(b), "d%d n%lldx%lldx%lld t%d o%d bc%d v%d V%d", c->d, (long long)c->n[0], (long long)c->n[1],
           (long long)c->n[2], c->dtype, c->order, c->bc, c->variant, c->V ? 1 : 0);
  return b;
}

bool tune_file_lookup(const std::string& key, int* cfg) {
  const char* path = getenv("NLSE_TUNE_CACHE");
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[256];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    char* eq = strrchr(line, '=');
    if (!eq) continue;
    *eq = 0;
    if (key == line) { *cfg = atoi(eq + 1); found = true; }
  }
  fclose(f);
  return found;
}

void tune_file_store(const std::string& key, int cfg) {
  const char* path = getenv("NLSE_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s=%d\n", key.c_str(), cfg);
  fclose(f);
}
}  // namespace

int nlse_autotune(nlse_t c, int* best_tile_cfg, float* best_ms) {
  if (!c) return fail(NLSE_EINVAL, "NULL context");
  if (c->d == 1 || c->variant == 0 || c->variant == 3) {   // nothing tiled to tune
    if (best_tile_cfg) *best_tile_cfg = -1;
    if (best_ms) *best_ms = 0.f;
    return NLSE_OK;
  }
  const std::string key = tune_key(c);
  int cfg = -1;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) cfg = it->second;
  }
  float best = 0.f;
  if (cfg < 0 && tune_file_lookup(key, &cfg)) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = cfg;
  }
  if (cfg < 0) {
    // time stage 2 (the heaviest stage) for every tile; stage 1 fills its inputs.
    // Neither stage writes Psi.
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved = c->tile_cfg;
    best = 1e30f;
    cudaError_t e = cudaSuccess;
    if (c->dtype == NLSE_C64_ACC64)
      e = launch_round_master((const double2*)c->psi, (float2*)c->at(c->lay.pn32), c->total, c->stream);
    if (e == cudaSuccess && c->exact()) e = update_fix(c, c->psi, c->stream);
    for (int t = 0; t < 4 && e == cudaSuccess; ++t) {
      c->tile_cfg = t;
      e = launch_stage_any(c, 1, 1e-12, c->stream);
      if (e == cudaSuccess) e = launch_stage_any(c, 2, 1e-12, c->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
      for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_stage_any(c, 2, 1e-12, c->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms / 3 < best) { best = ms / 3; cfg = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tile_cfg = saved;
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = cfg;
    tune_file_store(key, cfg);
  }
  c->tile_cfg = cfg;
  drop_graph(c);
  if (best_tile_cfg) *best_tile_cfg = cfg;
  if (best_ms) *best_ms = best;
  return NLSE_OK;
}

int nlse_debug_set(nlse_t c, int key, long long value) {
  if (!c) return fail(NLSE_EINVAL, "NULL context");
  switch (key) {
    case NLSE_DEBUG_SPIN_LIMIT:
      if (value <= 0) return fail(NLSE_EINVAL, "spin limit must be > 0");
      c->spin_limit = value;
      break;
    case NLSE_DEBUG_EXTRA_TX:
      if (value < 0 || value > (1 << 20) || value % 16) return fail(NLSE_EINVAL, "extra_tx must be 0..2^20, multiple of 16");
      c->extra_tx = (unsigned int)value;
      break;
    case NLSE_DEBUG_FIX_OFFSET:
      if (value < -64 || value > 64) return fail(NLSE_EINVAL, "fix offset must be -64..64");
      c->fix_offset = (int)value;
      break;
    default:
      return fail(NLSE_EINVAL, "unknown debug key");
  }
  drop_graph(c);
  return NLSE_OK;
}

int nlse_sync(nlse_t c) {
  if (!c) return fail(NLSE_EINVAL, "NULL context");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pending error");
  return read_status(c);
}

int nlse_destroy(nlse_t c) {
  if (!c) return NLSE_OK;
  drop_graph(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  for (int i = 0; i < 2; ++i) {
    if (c->side_yx[i]) cudaStreamDestroy(c->side_yx[i]);
    if (c->ev_join_yx[i]) cudaEventDestroy(c->ev_join_yx[i]);
  }
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
  return NLSE_OK;
}

}  // extern "C"
