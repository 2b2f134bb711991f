// Two RK4 stages per pass (temporal blocking) for the FP32 form on 3D grids.
//
// Eq. RK4_GPU streams the whole grid through HBM once per stage: stage 1 reads
// Psi^n and writes K_tot and Psi_tmp, stage 2 reads them back, and so on (152
// bytes per site and step with V).  Here a pass computes two consecutive
// stages, (1, 2) or (3, 4), in one sweep: the first stage's output for a tile
// plus a two-cell halo stays in shared memory and feeds the second stage's
// stencil directly, so the intermediate state never goes to HBM.
//
// A CTA owns a TX x TY tile of (x, y) columns and marches along z.  The first
// stage's input arrives by one TMA load per plane with a four-cell halo (the
// second stage's stencil reaches two cells, and each of those values needs a
// stencil reaching two more) into a ring of 5 + P slots.  For each plane z1
// the first stage is evaluated on the tile plus a two-cell halo (every site
// of that region at least two cells from every wall: no wall logic), its
// result Psi_mid = Psi^n + c1 F goes into a ring of five planes, and the
// second stage then runs on the tile's sites of plane z1 - 2.  Every site's
// arithmetic is the stage-streaming kernels' (a_lap_body, rk_apply), in the
// same order, so the result is bit-for-bit theirs.
//
// Ownership of the writes (distances are to the nearest wall along each axis):
//   R2: every index in [4, N-5]                 the second stage's outputs
//   R1 \ R2: z, y in [2, N-3], x in [4, Nx-5]   the first stage's outputs (these
//        sites' second stage belongs to the shell kernel)
//   R2 within five cells of a wall              also Psi_mid, which the second
//        stage's shell kernel reads as its stencil input
// The first stage's shell (z, y walls one layer, x walls three) and the
// second stage's shell (three layers at every wall) are the slab kernels.
//
// Pass (3, 4) writes Psi^{n+1} into the other buffer of a ping-pong pair,
// because its first stage reads Psi^n at halo sites that neighbouring CTAs
// own (stage 4 of Eq. RK4_GPU otherwise updates Psi in place).
#pragma once
#include "stage_slab.cuh"
#include "stage_tma.cuh"

namespace nlse {

template <int TX, int TY>
struct FusedGeom {
  static constexpr int W4 = TX + 8, H4 = TY + 8, PS4 = W4 * H4;   // input plane with a four-cell halo
  static constexpr int W2 = TX + 4, H2 = TY + 4, PS2 = W2 * H2;   // first-stage region: two-cell halo
  static constexpr uint32_t kBytes = PS4 * sizeof(float2);
  static constexpr uint32_t kSlot = (kBytes + 127u) / 128u * 128u;
  static constexpr uint32_t kMid = (PS2 * sizeof(float2) + 127u) / 128u * 128u;
  static constexpr uint32_t kK = (TX * TY * sizeof(float2) + 127u) / 128u * 128u;
};

// S1 = the first stage of the pass (1 or 3); the second is S1 + 1.
// A1, A2: the two stages' arguments as the stage-streaming path builds them
// (A2.master: where stage 4 writes Psi^{n+1}; A2.psin / load of the master
// read Psi^n from A1.psin).
template <int ORDER, int S1, int TX, int TYT, int RY, int P>
__global__ void __launch_bounds__(TX* TYT, 2) k_stage3d_fused(const StageArgs<P32> A1, const StageArgs<P32> A2,
                                                              const __grid_constant__ CUtensorMap tm, int zc,
                                                              long long spin_limit, uint32_t extra_tx) {
  constexpr int TY = TYT * RY, NT = TX * TYT, RS = 5 + P;
  using G = FusedGeom<TX, TY>;
  extern __shared__ __align__(128) unsigned char fused_smem[];
  unsigned char* slots = fused_smem;                                            // RS input planes
  float2* mid = reinterpret_cast<float2*>(fused_smem + RS * G::kSlot);          // 5 first-stage planes
  float2* kr = reinterpret_cast<float2*>(fused_smem + RS * G::kSlot + 5 * G::kMid);   // 3 planes of K at the tile
  uint64_t* bars = reinterpret_cast<uint64_t*>(fused_smem + RS * G::kSlot + 5 * G::kMid + 3 * G::kK);
  const Field<P32>& f = A1.f;
  const int nz = f.n[0], ny = f.n[1], nx = f.n[2];
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int zb = 2 + blockIdx.z * zc;               // tile planes [zb, ze) of the first stage's range [2, nz-3]
  const int ze = min(zb + zc, nz - 2);
  const int z1b = max(zb - 2, 2), z1e = min(ze + 2, nz - 2);   // first-stage planes [z1b, z1e)
  const int jb = z1b - 2, jl = z1e + 1;             // input planes [jb, jl] are loaded
  const int64_t plane = (int64_t)ny * nx;
  const bool with_v = f.V != nullptr;

  if (tid == 0) {
    for (int s = 0; s < RS; ++s) mbar_init(smem_u32(bars + s), 1);
    mbar_fence_init();
  }
  __syncthreads();
  int islot = 0, issued = jb - 1;
  auto issue = [&](int j) {
    mbar_expect_tx(smem_u32(bars + islot), G::kBytes + extra_tx);
    tma_load_3d(smem_u32(slots + islot * G::kSlot), &tm, 2 * (x0 - 4), y0 - 4, j, smem_u32(bars + islot));
    islot = (islot + 1 == RS) ? 0 : islot + 1;
    issued = j;
  };
  if (tid == 0)
    for (int j = jb; j < jb + RS && j <= jl; ++j) issue(j);

  // input planes z1-2 .. z1+2 of the first plane
  const float2* pl[5];
  int wslot = 0;
  uint32_t wpar = 0;
  bool late = false;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    late |= !mbar_wait_bounded(smem_u32(bars + wslot), wpar, spin_limit);
    pl[d] = reinterpret_cast<const float2*>(slots + wslot * G::kSlot);
    if (++wslot == RS) { wslot = 0; wpar ^= 1u; }
  }
  auto in_deep = [](int i, int n, int d) { return i >= d && i <= n - 1 - d; };
  // ring slots by plane number: first-stage plane z in mid slot (z - z1b) mod 5, its tile K in slot mod 3
  auto mslot = [&](int z) { const int q = (z - z1b) % 5; return mid + (q < 0 ? q + 5 : q) * (G::kMid / sizeof(float2)); };
  auto kslot = [&](int z) { const int q = (z - z1b) % 3; return kr + (q < 0 ? q + 3 : q) * (G::kK / sizeof(float2)); };

  // This thread's first-stage sites (the same (x, y) on every plane): element e = tid + k NT of the
  // tile-plus-halo region, needed when at least two cells from the x and y walls.
  constexpr int NS1 = (G::PS2 + NT - 1) / NT;
  int s1o[NS1], s1k[NS1];         // element in the input plane; tile position (cy TX + cx) or -1
  int64_t s1c[NS1];               // column offset gy nx + gx
  bool s1ok[NS1];
#pragma unroll
  for (int k = 0; k < NS1; ++k) {
    const int e = tid + k * NT;
    const int ry = e / G::W2, rx = e - ry * G::W2;
    const int gx = x0 - 2 + rx, gy = y0 - 2 + ry;
    s1ok[k] = e < G::PS2 && in_deep(gx, nx, 2) && in_deep(gy, ny, 2);
    s1o[k] = (ry + 2) * G::W4 + rx + 2;
    const int cx = rx - 2, cy = ry - 2;
    s1k[k] = (cx >= 0 && cx < TX && cy >= 0 && cy < TY) ? cy * TX + cx : -1;
    s1c[k] = (int64_t)gy * nx + gx;
  }
  // the pointwise operands the first stage reads from global memory, one plane ahead
  float v1[NS1], v1n[NS1];
  float2 pn1[NS1], pn1n[NS1], k1[NS1], k1n[NS1];
  auto load1 = [&](int z, float* v, float2* pn, float2* kk) {
#pragma unroll
    for (int k = 0; k < NS1; ++k) {
      if (!s1ok[k] || z >= z1e) continue;
      const int64_t c = z * plane + s1c[k];
      v[k] = with_v ? __ldg(f.V + c) : 0.f;
      if (S1 == 3) {
        pn[k] = __ldg(A1.psin + c);
        if (s1k[k] >= 0) kk[k] = __ldg(A1.ktot + c);
      }
    }
  };
  // the second stage's sites and their operands (V; Psi^n for stage 4), one plane ahead
  float v2[RY], v2n[RY];
  float2 pn2[RY], pn2n[RY];
  auto load2 = [&](int z) {
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y + r * TYT;
      if (!(z >= zb && z < ze && in_deep(z, nz, 4) && in_deep(gx, nx, 4) && in_deep(gy, ny, 4))) continue;
      const int64_t c = z * plane + (int64_t)gy * nx + gx;
      v2n[r] = with_v ? __ldg(f.V + c) : 0.f;
      if (S1 == 3) pn2n[r] = __ldg(A1.psin + c);
    }
  };
  load1(z1b, v1, pn1, k1);
  load2(z1b - 2);
#pragma unroll
  for (int r = 0; r < RY; ++r) { v2[r] = v2n[r]; pn2[r] = pn2n[r]; }

  bool aborted = false;
  // iteration z1: the first stage at plane z1 (while z1 < z1e), then the second stage at plane z1 - 2
  for (int z1 = z1b; z1 < ze + 2; ++z1) {
    load1(z1 + 1, v1n, pn1n, k1n);   // next plane's operands in flight during this plane's work
    load2(z1 - 1);
    // ---- first stage at plane z1, tile + two-cell halo ----
    if (z1 < z1e) {
      late |= !mbar_wait_bounded(smem_u32(bars + wslot), wpar, spin_limit);
      pl[4] = reinterpret_cast<const float2*>(slots + wslot * G::kSlot);
      if (++wslot == RS) { wslot = 0; wpar ^= 1u; }
      float2* mplane = mslot(z1);
      float2* kplane = kslot(z1);
#pragma unroll
      for (int k = 0; k < NS1; ++k) {
        if (!s1ok[k] || late) continue;
        const int e = tid + k * NT;
        const int64_t c = z1 * plane + s1c[k];
        SAcc3<P32> acc;
#pragma unroll
        for (int d = 0; d < 5; ++d) acc.p[d] = pl[d];
        acc.w = G::W4;
        acc.o = s1o[k];
        const int idx[3] = {z1, 0, 0};   // unused by the wall-free stencil
        const float2 pc = acc.at0();
        const float Nc = fmaf(f.s, norm2(pc), -v1[k]);
        const float2 aL = a_lap_body<P32, 3, ORDER, SAcc3<P32>, false>(f, acc, idx, c, pc, Nc);
        const float2 F = {-fmaf(Nc, pc.y, aL.y), fmaf(Nc, pc.x, aL.x)};
        const float2 pn = (S1 == 1) ? pc : pn1[k];     // Psi^n
        mplane[e] = make_float2(fmaf(A1.dtc, F.x, pn.x), fmaf(A1.dtc, F.y, pn.y));
        if (s1k[k] >= 0) {     // a tile site: keep its K for the second stage
          float2 K = F;
          if (S1 == 3) K = make_float2(fmaf(2.f, F.x, k1[k].x), fmaf(2.f, F.y, k1[k].y));
          kplane[s1k[k]] = K;
        }
      }
    }
    if (__syncthreads_or(late)) {
      aborted = true;
      break;
    }
    // ---- second stage at plane z2 = z1 - 2 (first-stage planes z2-2 .. z2+2 are in the ring) ----
    const int z2 = z1 - 2;
    if (z2 >= zb && z2 < ze) {
      const float2* mp[5];
#pragma unroll
      for (int d = 0; d < 5; ++d) mp[d] = mslot(z2 - 2 + d);
      const float2* kplane = kslot(z2);
      const bool r2z = in_deep(z2, nz, 4), nearz = !in_deep(z2, nz, 6);
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        const int cy = threadIdx.y + r * TYT, cx = threadIdx.x;
        const int gx = x0 + cx, gy = y0 + cy;
        if (!(in_deep(gx, nx, 4) && in_deep(gy, ny, 2))) continue;   // first-stage shell or outside
        const int64_t c = z2 * plane + (int64_t)gy * nx + gx;
        const int o2 = (cy + 2) * G::W2 + cx + 2;
        const float2 K = kplane[cy * TX + cx];
        if (!(r2z && in_deep(gx, nx, 4) && in_deep(gy, ny, 4))) {
          // R1 \ R2: the first stage's outputs; the second stage is the shell's
          A1.ktot[c] = K;
          A1.out[c] = mp[2][o2];
          continue;
        }
        if (nearz || !in_deep(gx, nx, 6) || !in_deep(gy, ny, 6)) A1.out[c] = mp[2][o2];   // the shell's stencil input
        SAcc3<P32> acc;
#pragma unroll
        for (int d = 0; d < 5; ++d) acc.p[d] = mp[d];
        acc.w = G::W2;
        acc.o = o2;
        const int idx[3] = {z2, gy, gx};
        PointVals<P32> pv;
        pv.v = v2[r];
        const float2 pc = acc.at0();
        const float Nc = fmaf(A2.f.s, norm2(pc), -pv.v);
        const float2 aL = a_lap_body<P32, 3, ORDER, SAcc3<P32>, false>(A2.f, acc, idx, c, pc, Nc);
        pv.K = K;
        if (S1 == 1) pv.pn = pl[0][(cy + 4) * G::W4 + cx + 4];   // Psi^n at plane z2 = z1 - 2: input ring plane 0
        else pv.mst = pn2[r];
        rk_apply<P32, S1 + 1>(A2, c, {-fmaf(Nc, pc.y, aL.y), fmaf(Nc, pc.x, aL.x)}, pv);
      }
    }
    if (__syncthreads_or(late)) {
      aborted = true;
      break;
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) pl[d] = pl[d + 1];     // pl[0] is plane z1 - 1 from here on
#pragma unroll
    for (int k = 0; k < NS1; ++k) { v1[k] = v1n[k]; pn1[k] = pn1n[k]; k1[k] = k1n[k]; }
#pragma unroll
    for (int r = 0; r < RY; ++r) { v2[r] = v2n[r]; pn2[r] = pn2n[r]; }
    if (tid == 0 && z1 < z1e && issued < jl) issue(issued + 1);   // the slot of plane z1 - 2 is free now
  }
  if (aborted && tid == 0) {
    atomicOr(A1.flag, kFlagTimeout);
    for (int j = max(jb, issued - RS + 1); j <= issued; ++j) {
      const int q = j - jb;
      mbar_wait_bounded(smem_u32(bars + q % RS), uint32_t((q / RS) & 1), spin_limit);
    }
  }
}

// Tile of the fused kernel: 64 x 8 sites, 256 threads (two rows each).
constexpr int kFusedTX = 64, kFusedTYT = 4, kFusedRY = 2, kFusedP = 2;
static_assert(kFusedBoxX == 2 * (kFusedTX + 8) && kFusedBoxY == kFusedTYT * kFusedRY + 8, "TMA box of the fused kernel");

inline size_t fused_smem_bytes() {
  using G = FusedGeom<kFusedTX, kFusedTYT * kFusedRY>;
  return (5 + kFusedP) * G::kSlot + 5 * G::kMid + 3 * G::kK + (5 + kFusedP) * sizeof(uint64_t);
}

// The fused kernel's planes: the first stage's range [2, Nz-3] in chunks.
template <int ORDER, int S1>
cudaError_t launch_fused_kernel(const StageArgs<P32>& A1, const StageArgs<P32>& A2, const CUtensorMap* tm,
                                long long spin_limit, uint32_t extra_tx, cudaStream_t stream) {
  constexpr int TX = kFusedTX, TY = kFusedTYT * kFusedRY;
  const int nz = A1.f.n[0], ny = A1.f.n[1], nx = A1.f.n[2];
  const int tiles = ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY);
  const int planes = nz - 4;
  const size_t smem = fused_smem_bytes();
  auto kern = k_stage3d_fused<ORDER, S1, TX, kFusedTYT, kFusedRY, kFusedP>;
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    per_sm = resident_per_sm(kern, TX * kFusedTYT, smem);
  }
  // six extra planes: a chunk's rings fill and drain
  int nzc = z_chunks(tiles, planes, per_sm, 6);
  const int zc = (planes + nzc - 1) / nzc;
  nzc = (planes + zc - 1) / zc;
  dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, nzc);
  kern<<<grid, dim3(TX, kFusedTYT), smem, stream>>>(A1, A2, *tm, zc, spin_limit, extra_tx);
  return cudaGetLastError();
}

// The second stage's shell: three site layers at every wall, as slabs.
//   z walls  z in {1,2,3, Nz-4..Nz-2},  y in [1, Ny-2], x in [1, Nx-2]
//   y walls  z in [4, Nz-5],  y in {1,2,3, Ny-4..Ny-2}, x in [1, Nx-2]
//   x walls  z in [4, Nz-5],  y in [4, Ny-5], x in {1,2,3, Nx-4..Nx-2}
template <int ORDER>
cudaError_t launch_shell_slabs3(const StageArgs<P32>& A, cudaStream_t stream) {
  const int* n = A.f.n;
  cudaError_t e;
  if ((e = launch_slab<P32, ORDER, false, 1, 0, 2, 3>(A, SlabRange{1, n[1] - 2, 1, n[2] - 2}, stream)) != cudaSuccess)
    return e;
  if ((e = launch_slab<P32, ORDER, false, 0, 1, 2, 3>(A, SlabRange{4, n[0] - 5, 1, n[2] - 2}, stream)) != cudaSuccess)
    return e;
  return launch_slab<P32, ORDER, false, 0, 2, 1, 3>(A, SlabRange{4, n[0] - 5, 4, n[1] - 5}, stream);
}

// Grids the fused path takes: every extent >= 16 (the shells' layers must not
// meet), and the TMA layout (checked by the caller).
inline bool fused_ok(const int* n) { return n[0] >= 16 && n[1] >= 16 && n[2] >= 16; }

}  // namespace nlse
