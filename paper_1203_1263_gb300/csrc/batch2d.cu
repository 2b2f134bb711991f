// Batched form: many independent 2D runs of uneven size and parameters
// advanced together, one launch per stage for all of them.
//
// Each run has its own grid (Ny, Nx), spacing, a, s, potential, boundary,
// order and time step.  A device table holds, per run, the stage arguments
// of the four RK4 stages (the same StageArgs the single-run kernels use); a
// work list enumerates (run, tile) items covering every run's deep interior,
// and a second list covers every run's wall shell in chunks of at most 256
// sites.  The deep kernel is persistent: a grid of a few CTAs per SM walks
// the item list, loads each tile with its 2-cell halo into shared memory and
// computes it with the per-site code of every other kernel; the shell kernel
// runs on a side stream at the same time.  Results are therefore bit-for-bit
// those of integrating each run alone with the tiled kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/nlse.h"
#include "nlse_internal.h"
#include "stage_generic.cuh"
#include "stage_tiled.cuh"

namespace nlse {
void record_last_error(const char* msg);
}

using namespace nlse;

namespace {

struct BatchRun {
  StageArgs<P32> A[4];   // stages 1..4
  int order;
  int pad[3];
};

struct DeepItem {
  int run, tx, ty, pad;
};

struct ShellItem {
  int run, start, count, pad;
};

constexpr int kShellChunk = 256;
constexpr int kGraphSteps = 16;

int bfail(int code, const char* msg) {
  nlse::record_last_error(msg);
  return code;
}

template <int ORDER, int TX, int TY>
__device__ __forceinline__ void batch_tile(const StageArgs<P32>& A, int tx, int ty, float2* tile) {
  constexpr int W = TX + 4, H = TY + 4, PS = W * H, NT = TX * TY, NPER = (PS + NT - 1) / NT;
  const Field<P32>& f = A.f;
  const int ny = f.n[0], nx = f.n[1];
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int x0 = tx * TX, y0 = ty * TY;
  const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
  const bool deep = gx >= 2 && gx <= nx - 3 && gy >= 2 && gy <= ny - 3;
  const int64_t c = (int64_t)gy * nx + gx;
  // the site's pointwise operands are requested first, so that their latency
  // overlaps the tile's
  PointVals<P32> pv;
  if (deep) pv = load_point<P32>(A, c, f.V != nullptr);
#pragma unroll
  for (int i = 0; i < NPER; ++i) {
    const int e = tid + i * NT;
    if (e < PS) {
      const int r = e / W, q = e - r * W;
      const int gy = y0 - 2 + r, gx = x0 - 2 + q;
      tile[e] = (gy >= 0 && gy < ny && gx >= 0 && gx < nx) ? f.in[(int64_t)gy * nx + gx] : float2{0.f, 0.f};
    }
  }
  __syncthreads();
  if (deep) {
    const int idx[2] = {gy, gx};
    SAcc2<P32> acc;
    acc.p = tile;
    acc.w = W;
    acc.o = (threadIdx.y + 2) * W + threadIdx.x + 2;
    const float2 pc = acc.at0();
    const float Nc = fmaf(f.s, norm2(pc), -pv.v);
    const float2 aL = a_lap_body<P32, 2, ORDER, SAcc2<P32>, false>(f, acc, idx, c, pc, Nc);
    rk_apply<P32>(A, c, {-fmaf(Nc, pc.y, aL.y), fmaf(Nc, pc.x, aL.x)}, pv);
  }
  __syncthreads();   // the tile is reused by the next item
}

template <int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_batch2d_deep(const BatchRun* __restrict__ runs,
                                                        const DeepItem* __restrict__ items, int nitems, int stage) {
  __shared__ __align__(16) float2 tile[(TX + 4) * (TY + 4)];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const DeepItem w = items[it];
    const BatchRun& R = runs[w.run];
    const StageArgs<P32>& A = R.A[stage - 1];
    if (R.order == 4) batch_tile<4, TX, TY>(A, w.tx, w.ty, tile);
    else batch_tile<2, TX, TY>(A, w.tx, w.ty, tile);
  }
}

__global__ void __launch_bounds__(kShellChunk) k_batch2d_shell(const BatchRun* __restrict__ runs,
                                                               const ShellItem* __restrict__ items, int stage) {
  const ShellItem w = items[blockIdx.x];
  if ((int)threadIdx.x >= w.count) return;
  const BatchRun& R = runs[w.run];
  const StageArgs<P32>& A = R.A[stage - 1];
  int idx[2];
  const int64_t c = shell_decode<P32, 2, uint32_t>(A.f, uint32_t(w.start + threadIdx.x), idx);
  const GAcc<P32, 2> acc(A.f, c);
  if (R.order == 4) process_site<P32, 2, 4, false>(A, acc, idx, c);
  else process_site<P32, 2, 2, false>(A, acc, idx, c);
}

// Run-table and work-list layout inside the caller's workspace.
struct BatchLayout {
  size_t runs_off, deep_off, shell_off, fields_off, total;
  int ndeep, nshell;
  std::vector<size_t> field_off;   // per run: K_tot, Psi_tmp, Psi_out (3 x 8 B x sites)
};

void tile_dims(int tile_cfg, int* tx, int* ty) { tma_tile_shape(tile_cfg < 0 ? 0 : tile_cfg, tx, ty); }

bool layout_batch(int nruns, const nlse_run_desc* runs, int tile_cfg, BatchLayout* L) {
  int tx, ty;
  tile_dims(tile_cfg, &tx, &ty);
  size_t off = 256;   // bytes 0..255: the status word, at the same place for every tile shape
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  L->runs_off = off;
  off = al(off + sizeof(BatchRun) * nruns);
  int64_t nd = 0, ns = 0;
  for (int r = 0; r < nruns; ++r) {
    const int64_t ny = runs[r].n[0], nx = runs[r].n[1];
    if (ny < 3 || nx < 3) return false;
    if (ny > 4 && nx > 4) nd += ((nx + tx - 1) / tx) * ((ny + ty - 1) / ty);
    const int m[2] = {int(ny - 2), int(nx - 2)};
    ns += (shell_count(2, m) + kShellChunk - 1) / kShellChunk;
  }
  if (nd > (1ll << 30) || ns > (1ll << 30)) return false;
  L->ndeep = int(nd);
  L->nshell = int(ns);
  L->deep_off = off;
  off = al(off + sizeof(DeepItem) * nd);
  L->shell_off = off;
  off = al(off + sizeof(ShellItem) * ns);
  L->fields_off = off;
  L->field_off.resize(nruns);
  for (int r = 0; r < nruns; ++r) {
    L->field_off[r] = off;
    off = al(off + 3 * sizeof(float2) * size_t(runs[r].n[0] * runs[r].n[1]));
  }
  L->total = al(off);
  return true;
}

}  // namespace

struct nlse_batch {
  int nruns;
  std::vector<nlse_run_desc> desc;
  char* ws;
  BatchLayout lay;
  cudaStream_t stream, side, cap;
  cudaEvent_t ev_fork, ev_join;
  cudaGraphExec_t exec;
  int tile_cfg;
  unsigned int* flag() const { return (unsigned int*)ws; }   // fixed: the layout after it depends on the tile shape
};

namespace {

template <int TX, int TY>
cudaError_t launch_deep(const nlse_batch* b, int stage, cudaStream_t st) {
  if (b->lay.ndeep == 0) return cudaSuccess;
  // one wave of persistent CTAs: as many as fit on every SM at once for this tile shape
  static int per_sm = 0, sms = 0;
  if (per_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch2d_deep<TX, TY>, TX * TY, 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
  }
  int grid = sms * per_sm;
  if (grid > b->lay.ndeep) grid = b->lay.ndeep;
  k_batch2d_deep<TX, TY><<<grid, dim3(TX, TY), 0, st>>>((const BatchRun*)(b->ws + b->lay.runs_off),
                                                         (const DeepItem*)(b->ws + b->lay.deep_off), b->lay.ndeep,
                                                         stage);
  return cudaGetLastError();
}

cudaError_t launch_batch_stage(const nlse_batch* b, int stage, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaEventRecord(b->ev_fork, st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(b->side, b->ev_fork, 0)) != cudaSuccess) return e;
  if (b->lay.nshell > 0) {
    k_batch2d_shell<<<b->lay.nshell, kShellChunk, 0, b->side>>>((const BatchRun*)(b->ws + b->lay.runs_off),
                                                                  (const ShellItem*)(b->ws + b->lay.shell_off), stage);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = cudaEventRecord(b->ev_join, b->side)) != cudaSuccess) return e;
  switch (b->tile_cfg < 0 ? 0 : b->tile_cfg) {
    case 0: e = launch_deep<32, 8>(b, stage, st); break;
    case 1: e = launch_deep<64, 4>(b, stage, st); break;
    case 2: e = launch_deep<32, 16>(b, stage, st); break;
    default: e = launch_deep<64, 8>(b, stage, st); break;
  }
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(st, b->ev_join, 0);
}

cudaError_t launch_batch_step(const nlse_batch* b, cudaStream_t st) {
  for (int s = 1; s <= 4; ++s) {
    cudaError_t e = launch_batch_stage(b, s, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Build the run table and work lists on the host and copy them into the workspace.
int upload_tables(nlse_batch* b) {
  int tx, ty;
  tile_dims(b->tile_cfg, &tx, &ty);
  std::vector<BatchRun> runs(b->nruns);
  std::vector<DeepItem> deep;
  std::vector<ShellItem> shell;
  deep.reserve(b->lay.ndeep);
  shell.reserve(b->lay.nshell);
  // work items of large runs first, so that the persistent CTAs run out of work together
  std::vector<int> order(b->nruns);
  for (int r = 0; r < b->nruns; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
    return b->desc[p].n[0] * b->desc[p].n[1] > b->desc[q].n[0] * b->desc[q].n[1];
  });
  for (int r : order) {
    const nlse_run_desc& d = b->desc[r];
    const int ny = int(d.n[0]), nx = int(d.n[1]);
    float2* base = (float2*)(b->ws + b->lay.field_off[r]);
    const int64_t sites = (int64_t)ny * nx;
    float2 *ktot = base, *ptmp = base + sites, *pout = base + 2 * sites;
    BatchRun& R = runs[r];
    memset(&R, 0, sizeof(R));
    R.order = d.order;
    const void* in[4] = {d.psi, ptmp, pout, ptmp};
    float2* outs[4] = {ptmp, pout, ptmp, nullptr};
    const double dtc[4] = {d.dt / 2.0, d.dt / 2.0, d.dt, d.dt / 6.0};
    for (int s = 0; s < 4; ++s) {
      StageArgs<P32>& A = R.A[s];
      Field<P32>& f = A.f;
      f.n[0] = ny; f.n[1] = nx; f.n[2] = 1;
      f.m[0] = ny - 2; f.m[1] = nx - 2; f.m[2] = 1;
      f.st[0] = nx; f.st[1] = 1; f.st[2] = 0;
      f.ninterior = (int64_t)(ny - 2) * (nx - 2);
      f.a = float(d.a);
      f.s = float(d.s);
      f.h2_over_a = float(d.h * d.h / d.a);
      f.cL = float(d.order == 4 ? d.a / (12.0 * d.h * d.h) : d.a / (d.h * d.h));
      f.tiny = 1e-30f;
      f.bc = d.bc;
      f.V = (const float*)d.V;
      f.in = (const float2*)in[s];
      A.psin = (const float2*)d.psi;
      A.ktot = ktot;
      A.out = outs[s];
      A.master = (float2*)d.psi;
      A.master_in = (const float2*)d.psi;   // Psi updated in place: stage 4 reads Psi^n where it writes
      A.dtc = float(dtc[s]);
      A.dt6 = d.dt / 6.0;
      A.stage = s + 1;
      A.flag = b->flag();
    }
    if (ny > 4 && nx > 4)
      for (int t_y = 0; t_y < (ny + ty - 1) / ty; ++t_y)
        for (int t_x = 0; t_x < (nx + tx - 1) / tx; ++t_x) deep.push_back({r, t_x, t_y, 0});
    const int m[2] = {ny - 2, nx - 2};
    const int64_t nsh = shell_count(2, m);
    for (int64_t s0 = 0; s0 < nsh; s0 += kShellChunk)
      shell.push_back({r, int(s0), int(std::min<int64_t>(kShellChunk, nsh - s0)), 0});
  }
  cudaError_t e = cudaMemcpyAsync(b->ws + b->lay.runs_off, runs.data(), sizeof(BatchRun) * runs.size(),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess && !deep.empty())
    e = cudaMemcpyAsync(b->ws + b->lay.deep_off, deep.data(), sizeof(DeepItem) * deep.size(), cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess && !shell.empty())
    e = cudaMemcpyAsync(b->ws + b->lay.shell_off, shell.data(), sizeof(ShellItem) * shell.size(),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(NLSE_ECUDA, cudaGetErrorString(e));
  return NLSE_OK;
}

void drop_graph(nlse_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
}

int validate(int nruns, const nlse_run_desc* runs) {
  if (nruns <= 0 || !runs) return bfail(NLSE_EINVAL, "need at least one run");
  for (int r = 0; r < nruns; ++r) {
    const nlse_run_desc& d = runs[r];
    if (d.n[0] < 3 || d.n[1] < 3 || d.n[0] > (1 << 20) || d.n[1] > (1 << 20))
      return bfail(NLSE_EINVAL, "every run needs 3 <= N <= 2^20 on both axes");
    if (!(d.h > 0) || !(d.a > 0) || !isfinite(d.s) || !(d.dt > 0)) return bfail(NLSE_EINVAL, "run h, a, dt must be > 0");
    if (d.order != 2 && d.order != 4) return bfail(NLSE_EINVAL, "run order must be 2 or 4");
    if (d.bc != NLSE_BC_DIRICHLET && d.bc != NLSE_BC_MSD && d.bc != NLSE_BC_L0)
      return bfail(NLSE_EINVAL, "run bc must be 0, 1 or 2");
    if (!d.psi || (uintptr_t)d.psi % 8) return bfail(NLSE_EINVAL, "run psi must be an 8-byte aligned device pointer");
    const double rho = (d.order == 4 ? 32.0 / 3.0 : 8.0) / (d.h * d.h);
    if (d.dt > 2.0 * sqrt(2.0) / (d.a * rho)) return bfail(NLSE_EUNSTABLE, "a run's dt exceeds its RK4 linear bound");
  }
  return NLSE_OK;
}

}  // namespace

extern "C" {

size_t nlse_batch_workspace_bytes(int nruns, const nlse_run_desc* runs) {
  if (validate(nruns, runs) != NLSE_OK) return 0;
  BatchLayout L;
  if (!layout_batch(nruns, runs, -1, &L)) return 0;
  size_t worst = L.total;
  for (int t = 0; t < 4; ++t) {   // room for any tile shape
    BatchLayout Lt;
    if (layout_batch(nruns, runs, t, &Lt)) worst = std::max(worst, Lt.total);
  }
  return worst;
}

int nlse_batch_create(nlse_batch_t* out, int nruns, const nlse_run_desc* runs, void* workspace, size_t ws_bytes,
                      void* stream) {
  if (!out) return bfail(NLSE_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(nruns, runs);
  if (rc != NLSE_OK) return rc;
  if (!workspace || (uintptr_t)workspace % 256) return bfail(NLSE_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < nlse_batch_workspace_bytes(nruns, runs)) return bfail(NLSE_ENOMEM, "workspace too small");
  nlse_batch* b = new nlse_batch();
  b->nruns = nruns;
  b->desc.assign(runs, runs + nruns);
  b->ws = (char*)workspace;
  b->stream = (cudaStream_t)stream;
  b->tile_cfg = -1;
  b->side = b->cap = nullptr;
  b->exec = nullptr;
  layout_batch(nruns, runs, b->tile_cfg, &b->lay);
  cudaError_t e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->flag(), 0, 256, b->stream);
  if (e != cudaSuccess) {
    nlse_batch_destroy(b);
    return bfail(NLSE_ECUDA, cudaGetErrorString(e));
  }
  rc = upload_tables(b);
  if (rc != NLSE_OK) {
    nlse_batch_destroy(b);
    return rc;
  }
  *out = b;
  return NLSE_OK;
}

int nlse_batch_set_tile(nlse_batch_t b, int tile_cfg) {
  if (!b) return bfail(NLSE_EINVAL, "NULL batch");
  if (tile_cfg < -1 || tile_cfg > 3) return bfail(NLSE_EINVAL, "tile_cfg must be -1..3");
  b->tile_cfg = tile_cfg;
  layout_batch(b->nruns, b->desc.data(), tile_cfg, &b->lay);
  drop_graph(b);
  return upload_tables(b);
}

int nlse_batch_step(nlse_batch_t b, int64_t nsteps) {
  if (!b) return bfail(NLSE_EINVAL, "NULL batch");
  if (nsteps < 0) return bfail(NLSE_EINVAL, "nsteps < 0");
  cudaError_t e = cudaSuccess;
  int64_t left = nsteps;
  if (nsteps >= kGraphSteps) {
    if (!b->exec) {
      e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
      cudaError_t le = cudaSuccess;
      for (int i = 0; i < kGraphSteps && le == cudaSuccess && e == cudaSuccess; ++i) le = launch_batch_step(b, b->cap);
      cudaGraph_t g = nullptr;
      cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
      if (e == cudaSuccess) e = (le != cudaSuccess) ? le : ee;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->exec = nullptr;
        return bfail(NLSE_ECUDA, cudaGetErrorString(e));
      }
    }
    for (; left >= kGraphSteps && e == cudaSuccess; left -= kGraphSteps) e = cudaGraphLaunch(b->exec, b->stream);
  }
  for (; left > 0 && e == cudaSuccess; --left) e = launch_batch_step(b, b->stream);
  if (e != cudaSuccess) return bfail(NLSE_ECUDA, cudaGetErrorString(e));
  return NLSE_OK;
}

int nlse_batch_sync(nlse_batch_t b) {
  if (!b) return bfail(NLSE_EINVAL, "NULL batch");
  unsigned int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, b->flag(), sizeof(flag), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(NLSE_ECUDA, cudaGetErrorString(e));
  if (flag & 1u) return bfail(NLSE_ENONFINITE, "non-finite value in some run's Psi");
  return NLSE_OK;
}

int nlse_batch_autotune(nlse_batch_t b, int* best_tile_cfg, float* best_ms) {
  if (!b) return bfail(NLSE_EINVAL, "NULL batch");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float t_min[4] = {1e30f, 1e30f, 1e30f, 1e30f};
  int rc = NLSE_OK;
  // time stages 1-3 (none of them writes any run's Psi) for every tile shape,
  // twice in alternating order, after one untimed pass each; keep each shape's
  // fastest pass
  for (int pass = 0; pass < 3 && rc == NLSE_OK; ++pass) {
    for (int k = 0; k < 4 && rc == NLSE_OK; ++k) {
      const int t = (pass == 1) ? 3 - k : k;
      rc = nlse_batch_set_tile(b, t);
      if (rc != NLSE_OK) break;
      cudaError_t e = cudaEventRecord(e0, b->stream);
      for (int st = 1; st <= 3 && e == cudaSuccess; ++st) e = launch_batch_stage(b, st, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) rc = bfail(NLSE_ECUDA, cudaGetErrorString(e));
      else if (pass > 0 && ms < t_min[t]) t_min[t] = ms;   // pass 0 warms every shape up
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != NLSE_OK) return rc;
  int cfg = 0;
  for (int t = 1; t < 4; ++t)
    if (t_min[t] < t_min[cfg]) cfg = t;
  rc = nlse_batch_set_tile(b, cfg);
  if (best_tile_cfg) *best_tile_cfg = cfg;
  if (best_ms) *best_ms = t_min[cfg] / 3.f;
  return rc;
}

int nlse_batch_destroy(nlse_batch_t b) {
  if (!b) return NLSE_OK;
  drop_graph(b);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  delete b;
  return NLSE_OK;
}

}  // extern "C"
