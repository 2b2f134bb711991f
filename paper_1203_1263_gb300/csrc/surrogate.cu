// Learned surrogate: a residual convolutional network that advances a 2D
// complex state by one window of RK4 steps, trained and run on the GPU by the
// kernels in this file (BF16 tensor-core products with FP32 accumulation).
//
// Network (channels-last activations, H x W grid, batch nb):
//   h_{-1} = (Re psi, Im psi, |psi|^2 Re psi, |psi|^2 Im psi)    4 channels
//   z_l = conv3x3_{dil_l}(h_{l-1}) + b_l,  h_l = silu(z_l)       l = 0 .. L-2, C channels
//   y   = conv3x3_{dil_{L-1}}(h_{L-2}) + b_{L-1}                 2 channels
//   psi_out = psi_in + (y_0 + i y_1)
// with zero padding at the grid edges.  Parameters are FP32 masters; the
// products use BF16 copies.  Every convolution (forward, backward-data,
// weight-gradient) is an implicit GEMM, C[M x N] += A[M x K] B[K x N]:
//   forward        M = pixels, N = Cout, K = 9 Cin: A[p,(t,ci)] = h[p + d o_t, ci], B[(t,ci),co] = W[co,t,ci]
//   backward-data  M = pixels, N = Cin,  K = 9 Cout: A[p,(t,co)] = dz[p - d o_t, co], B[(t,co),ci] = W[co,t,ci]
//   weight-grad    M = Cout,   N = 9 Cin, K = pixels: A[co,p] = dz[p, co], B[p,(t,ci)] = h[p + d o_t, ci]
// Three kernel families compute them:
//   - tcgen05 (k_conv_tc, k_wgrad_tc): TMA-fed halo tiles in shared memory,
//     the nine taps as shifted descriptors over one tile, TMEM accumulators;
//     used for every layer whose channel counts fit (the 64-channel network
//     runs entirely on them);
//   - mma.sync.m16n8k16 with cp.async / ldmatrix staging (k_conv_fast), for
//     channel counts that are multiples of 8 (and for comparison);
//   - a scalar-gather mma.sync kernel (k_conv) for any other shape.
// Loss: mean squared error of psi_out against the target (Re and Im parts);
// optimiser: Adam.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "../../include/nlse.h"

namespace nlse {
void record_last_error(const char* msg);
void* tensor_map_encoder();
}

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kMaxLayers = 16;
constexpr int BM = 64, BN = 64, BK = 32, KPAD = 40;   // block tile; smem rows padded against bank conflicts
constexpr int kThreads = 128;                          // 4 warps, 2 x 2, each 32 x 32

int sfail(int code, const char* msg) {
  nlse::record_last_error(msg);
  return code;
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

struct Geo {
  int nb, H, W;
};

// tap t in 0..8 -> offsets (t/3 - 1, t%3 - 1)
__device__ __forceinline__ int tap_dy(int t) { return t / 3 - 1; }
__device__ __forceinline__ int tap_dx(int t) { return t % 3 - 1; }

// Value of activation `act` (channels-last, C channels) at pixel p shifted by (dy, dx), zero outside.
__device__ __forceinline__ float gather(const bf16* act, const Geo& g, int C, int64_t p, int dy, int dx, int c) {
  const int x = int(p % g.W), y = int((p / g.W) % g.H);
  const int yy = y + dy, xx = x + dx;
  if (yy < 0 || yy >= g.H || xx < 0 || xx >= g.W) return 0.f;
  return __bfloat162float(act[(p + (int64_t)dy * g.W + dx) * C + c]);
}

enum { MODE_FWD = 0, MODE_BWD_DATA = 1, MODE_WGRAD = 2 };

struct ConvArgs {
  Geo g;
  int cin, cout, dil;
  const bf16* x;        // forward / weight-grad input activation (Cin channels)
  const bf16* dz;       // backward: gradient w.r.t. the layer's pre-activation (Cout channels)
  const bf16* w;        // BF16 weights [Cout][9][Cin]
  const float* bias;    // forward
  float* z;             // forward: the last layer's output y (FP32), else nullptr
  bf16* h;              // forward: silu(z) out (BF16); nullptr for the last layer
  bf16* sd;             // forward (training): silu'(z) out (BF16), else nullptr
  const bf16* sdprev;   // backward-data: silu'(z) of the layer below (BF16), nullptr = none
  bf16* dzprev;         // backward-data: gradient w.r.t. the previous layer's pre-activation (BF16)
  float* dw;            // weight-grad: FP32 accumulation [Cout][9][Cin]
  int64_t kchunk;       // weight-grad: pixels per CTA
};

// One 64 x 64 output tile; the three modes differ only in the gathers and the epilogue.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_conv(const ConvArgs a) {
  __shared__ __align__(16) bf16 As[BM][KPAD];
  __shared__ __align__(16) bf16 Bs[BN][KPAD];   // stored N-major: Bs[n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;       // warp position in the 2 x 2 grid of 32 x 32 sub-tiles
  const Geo& g = a.g;
  const int64_t P = (int64_t)g.nb * g.H * g.W;
  int64_t M, N, K, m0, n0, k_begin, k_end;
  if (MODE == MODE_FWD) { M = P; N = a.cout; K = 9 * a.cin; }
  else if (MODE == MODE_BWD_DATA) { M = P; N = a.cin; K = 9 * a.cout; }
  else { M = a.cout; N = 9 * a.cin; K = P; }
  m0 = (int64_t)blockIdx.x * BM;
  n0 = (int64_t)blockIdx.y * BN;
  if (MODE == MODE_WGRAD) {
    k_begin = (int64_t)blockIdx.z * a.kchunk;
    k_end = k_begin + a.kchunk < K ? k_begin + a.kchunk : K;
  } else {
    k_begin = 0;
    k_end = K;
  }
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

  for (int64_t k0 = k_begin; k0 < k_end; k0 += BK) {
    // gather A (BM x BK) and B (BK x BN) into shared memory: 16 + 16 elements per thread
#pragma unroll 4
    for (int e = tid; e < BM * BK; e += kThreads) {
      const int r = e / BK, kk = e % BK;
      const int64_t m = m0 + r, k = k0 + kk;
      float v = 0.f;
      if (m < M && k < k_end) {
        if (MODE == MODE_FWD) {
          const int t = int(k / a.cin), ci = int(k % a.cin);
          v = gather(a.x, g, a.cin, m, a.dil * tap_dy(t), a.dil * tap_dx(t), ci);
        } else if (MODE == MODE_BWD_DATA) {
          const int t = int(k / a.cout), co = int(k % a.cout);
          v = gather(a.dz, g, a.cout, m, -a.dil * tap_dy(t), -a.dil * tap_dx(t), co);
        } else {
          v = __bfloat162float(a.dz[k * a.cout + m]);   // A[co, p] = dz[p, co]
        }
      }
      As[r][kk] = __float2bfloat16_rn(v);
    }
#pragma unroll 4
    for (int e = tid; e < BN * BK; e += kThreads) {
      const int c = e / BK, kk = e % BK;
      const int64_t n = n0 + c, k = k0 + kk;
      float v = 0.f;
      if (n < N && k < k_end) {
        if (MODE == MODE_FWD) {
          const int t = int(k / a.cin), ci = int(k % a.cin);
          v = __bfloat162float(a.w[((int64_t)n * 9 + t) * a.cin + ci]);
        } else if (MODE == MODE_BWD_DATA) {
          const int t = int(k / a.cout), co = int(k % a.cout);
          v = __bfloat162float(a.w[((int64_t)co * 9 + t) * a.cin + n]);
        } else {
          const int t = int(n / a.cin), ci = int(n % a.cin);
          v = gather(a.x, g, a.cin, k, a.dil * tap_dy(t), a.dil * tap_dx(t), ci);
        }
      }
      Bs[c][kk] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
      const int gr = lane >> 2, tg = lane & 3;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int row = wm * 32 + i * 16 + gr;
        af[i][0] = *reinterpret_cast<const uint32_t*>(&As[row][ks + tg * 2]);
        af[i][1] = *reinterpret_cast<const uint32_t*>(&As[row + 8][ks + tg * 2]);
        af[i][2] = *reinterpret_cast<const uint32_t*>(&As[row][ks + tg * 2 + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t*>(&As[row + 8][ks + tg * 2 + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int col = wn * 32 + j * 8 + gr;
        bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[col][ks + tg * 2]);
        bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[col][ks + tg * 2 + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }

  // epilogue: acc[i][j][r] is C[row, col] with row = wm*32 + i*16 + gr + (r>=2)*8, col = wn*32 + j*8 + tg*2 + (r&1)
  const int gr = lane >> 2, tg = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int64_t m = m0 + wm * 32 + i * 16 + gr + (r >= 2 ? 8 : 0);
        const int64_t n = n0 + wn * 32 + j * 8 + tg * 2 + (r & 1);
        if (m >= M || n >= N) continue;
        const float v = acc[i][j][r];
        if (MODE == MODE_FWD) {
          const float zv = v + a.bias[n];
          if (a.z) a.z[m * a.cout + n] = zv;
          if (a.sd) a.sd[m * a.cout + n] = __float2bfloat16_rn(dsilu(zv));
          if (a.h) a.h[m * a.cout + n] = __float2bfloat16_rn(silu(zv));
        } else if (MODE == MODE_BWD_DATA) {
          const float d = a.sdprev ? v * __bfloat162float(a.sdprev[m * a.cin + n]) : v;
          a.dzprev[m * a.cin + n] = __float2bfloat16_rn(d);
        } else {
          atomicAdd(&a.dw[m * (9 * a.cin) + n], v);   // dw[co][t][ci], n = t * Cin + ci
        }
      }
}

// ---------------------------------------------------------------------------
// Fast implicit-GEMM convolution for layers whose gathered channel counts are
// multiples of 8: operands move as 16-byte chunks (8 BF16 channels of one
// pixel, or 8 weights) with cp.async (zero-fill outside the grid) through a
// 3-stage shared-memory pipeline; fragments come from ldmatrix (transposed
// for the weight-gradient operands, whose natural layout is K-major rows).
// Warp grid WM x WN, each warp a 32 x 32 block of C; BK = 32.
// ---------------------------------------------------------------------------
constexpr int FBK = 32, FSTAGES = 3;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
               "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

// Pixel p = ((img * H) + y) * W + x shifted by (dy, dx): source pointer of channel chunk c0, or nullptr outside.
__device__ __forceinline__ const bf16* shifted(const bf16* act, const Geo& g, int C, int64_t p, int y, int x, int dy,
                                               int dx, int c0) {
  const int yy = y + dy, xx = x + dx;
  if (yy < 0 || yy >= g.H || xx < 0 || xx >= g.W) return nullptr;
  return act + (p + (int64_t)dy * g.W + dx) * C + c0;
}

template <int MODE, int WM, int WN>
__global__ void __launch_bounds__(WM * WN * 32) k_conv_fast(const ConvArgs a, const bf16* __restrict__ wt) {
  constexpr int NT = WM * WN * 32, BM_ = WM * 32, BN_ = WN * 32;
  constexpr bool KMAJOR = (MODE == MODE_WGRAD);      // operands stored [k][m] / [k][n]
  constexpr int AR = KMAJOR ? FBK : BM_, AC = KMAJOR ? BM_ + 8 : FBK + 8;
  constexpr int BR = KMAJOR ? FBK : BN_, BC = KMAJOR ? BN_ + 8 : FBK + 8;
  __shared__ __align__(128) bf16 As[FSTAGES][AR][AC];
  __shared__ __align__(128) bf16 Bs[FSTAGES][BR][BC];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp / WN, wn = warp % WN;
  const Geo& g = a.g;
  const int64_t P = (int64_t)g.nb * g.H * g.W;
  int64_t M, N, k_begin, k_end;
  if (MODE == MODE_FWD) { M = P; N = a.cout; k_begin = 0; k_end = 9 * a.cin; }
  else if (MODE == MODE_BWD_DATA) { M = P; N = a.cin; k_begin = 0; k_end = 9 * a.cout; }
  else {
    M = a.cout; N = 9 * a.cin;
    k_begin = (int64_t)blockIdx.z * a.kchunk;
    k_end = k_begin + a.kchunk < P ? k_begin + a.kchunk : P;
  }
  const int64_t m0 = (int64_t)blockIdx.x * BM_, n0 = (int64_t)blockIdx.y * BN_;

  // Per-thread copy assignments are fixed across k-tiles: the pixel rows of
  // the A chunks (FWD / BWD) and the tap / channel of the B^T chunks (WGRAD)
  // are decoded once; the WGRAD pixel rows advance by FBK per tile.
  constexpr int A_IT = KMAJOR ? 1 : (BM_ * 4) / NT;
  constexpr int B_IT = KMAJOR ? (FBK * (BN_ / 8)) / NT : 1;
  static_assert(KMAJOR || (BM_ * 4) % NT == 0, "A chunks per thread");
  static_assert(!KMAJOR || (FBK * (BN_ / 8)) % NT == 0, "B^T chunks per thread");
  int ay[A_IT], ax[A_IT];
  int64_t am[A_IT];
  int bdy = 0, bdx = 0, bc0 = 0;
  bool bval = false;
  int by[B_IT], bx[B_IT];
  if (!KMAJOR) {
#pragma unroll
    for (int i = 0; i < A_IT; ++i) {
      const int r = (tid + i * NT) >> 2;
      am[i] = m0 + r;
      const int64_t mm = am[i] < M ? am[i] : 0;
      ax[i] = int(mm % g.W);
      ay[i] = int((mm / g.W) % g.H);
    }
  } else {
    const int c = tid % (BN_ / 8);
    const int64_t n = n0 + 8 * c;
    bval = n < N;
    const int t = bval ? int(n / a.cin) : 0;
    bc0 = bval ? int(n - (int64_t)t * a.cin) : 0;
    bdy = a.dil * tap_dy(t);
    bdx = a.dil * tap_dx(t);
#pragma unroll
    for (int i = 0; i < B_IT; ++i) {
      const int64_t pp = k_begin + (tid + i * NT) / (BN_ / 8);
      bx[i] = int(pp % g.W);
      by[i] = int((pp / g.W) % g.H);
    }
  }

  // Issue the copies of k-tile k0 into stage st.
  auto load_tile = [&](int st, int64_t k0) {
    if (!KMAJOR) {
      // A: BM_ rows (pixels) x 4 chunks
      const int Cg = (MODE == MODE_FWD) ? a.cin : a.cout;
      const bf16* src_act = (MODE == MODE_FWD) ? a.x : a.dz;
      const int sgn = (MODE == MODE_FWD) ? 1 : -1;
#pragma unroll
      for (int i = 0; i < A_IT; ++i) {
        const int e = tid + i * NT;
        const int r = e >> 2, c = e & 3;
        const int k = int(k0) + 8 * c;
        const bf16* src = nullptr;
        if (am[i] < M && k < k_end) {
          const int t = k / Cg, c0 = k - t * Cg;
          src = shifted(src_act, g, Cg, am[i], ay[i], ax[i], sgn * a.dil * tap_dy(t), sgn * a.dil * tap_dx(t), c0);
        }
        cp16(&As[st][r][8 * c], src ? src : src_act, src != nullptr);
      }
      // B: BN_ rows (n) x 4 chunks; FWD from W[n][t][ci], BWD from WT[t][n][co]
#pragma unroll
      for (int e = tid; e < BN_ * 4; e += NT) {
        const int r = e >> 2, c = e & 3;
        const int64_t n = n0 + r;
        const int k = int(k0) + 8 * c;
        const bf16* src = nullptr;
        if (n < N && k < k_end) {
          if (MODE == MODE_FWD) src = a.w + n * 9 * a.cin + k;   // k = t * cin + ci
          else {
            const int t = k / a.cout, c0 = k - t * a.cout;
            src = wt + ((int64_t)t * a.cin + n) * a.cout + c0;
          }
        }
        cp16(&Bs[st][r][8 * c], src ? src : a.w, src != nullptr);
      }
    } else {
      // A^T: FBK rows (pixels) x BM_/8 chunks of dz[p][co]
#pragma unroll
      for (int e = tid; e < FBK * (BM_ / 8); e += NT) {
        const int r = e / (BM_ / 8), c = e % (BM_ / 8);
        const int64_t p = k0 + r, co = m0 + 8 * c;
        const bool v = p < k_end && co < M;
        cp16(&As[st][r][8 * c], v ? a.dz + p * a.cout + co : a.dz, v);
      }
      // B^T: FBK rows (pixels) x BN_/8 chunks of h[p + d o_t][ci], n = t * cin + ci
#pragma unroll
      for (int i = 0; i < B_IT; ++i) {
        const int e = tid + i * NT;
        const int r = e / (BN_ / 8), c = e % (BN_ / 8);
        const int64_t p = k0 + r;
        const bf16* src = (bval && p < k_end) ? shifted(a.x, g, a.cin, p, by[i], bx[i], bdy, bdx, bc0) : nullptr;
        cp16(&Bs[st][r][8 * c], src ? src : a.x, src != nullptr);
        // advance this row's pixel coordinates by FBK for the next tile
        int xx = bx[i] + FBK, yy = by[i];
        while (xx >= g.W) {
          xx -= g.W;
          if (++yy == g.H) yy = 0;
        }
        bx[i] = xx;
        by[i] = yy;
      }
    }
  };

  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

  const int64_t ntiles = (k_end - k_begin + FBK - 1) / FBK;
#pragma unroll
  for (int s0 = 0; s0 < FSTAGES - 1; ++s0) {
    if (s0 < ntiles) load_tile(s0, k_begin + (int64_t)s0 * FBK);
    cp_commit();
  }
  const int lr = lane & 7, lj = lane >> 3;
  for (int64_t kt = 0; kt < ntiles; ++kt) {
    cp_wait<FSTAGES - 2>();
    __syncthreads();
    {
      const int64_t nk = kt + FSTAGES - 1;
      if (nk < ntiles) load_tile(int(nk % FSTAGES), k_begin + nk * FBK);
      cp_commit();
    }
    const int st = int(kt % FSTAGES);
#pragma unroll
    for (int ks = 0; ks < FBK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int mb = wm * 32 + i * 16;
        if (!KMAJOR) ldsm_x4(af[i], &As[st][mb + (lj & 1) * 8 + lr][ks + (lj >> 1) * 8]);
        else ldsm_x4_t(af[i], &As[st][ks + (lj >> 1) * 8 + lr][mb + (lj & 1) * 8]);
      }
#pragma unroll
      for (int j2 = 0; j2 < 2; ++j2) {
        const int nb = wn * 32 + j2 * 16;
        uint32_t r4[4];
        if (!KMAJOR) ldsm_x4(r4, &Bs[st][nb + (lj >> 1) * 8 + lr][ks + (lj & 1) * 8]);
        else ldsm_x4_t(r4, &Bs[st][ks + (lj & 1) * 8 + lr][nb + (lj >> 1) * 8]);
        bfr[2 * j2][0] = r4[0];
        bfr[2 * j2][1] = r4[1];
        bfr[2 * j2 + 1][0] = r4[2];
        bfr[2 * j2 + 1][1] = r4[3];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bfr[j]);
    }
  }
  cp_wait<0>();

  // epilogue: acc[i][j][2h + q] is C[row, col], row = wm*32 + i*16 + gr + 8h, col = wn*32 + j*8 + 2tg + q
  const int gr = lane >> 2, tg = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int64_t m = m0 + wm * 32 + i * 16 + gr + 8 * hh;
        const int64_t n = n0 + wn * 32 + j * 8 + 2 * tg;
        if (m >= M) continue;
        const float v0 = acc[i][j][2 * hh], v1 = acc[i][j][2 * hh + 1];
        if (MODE == MODE_FWD) {
          if (n + 1 < N) {
            const float z0 = v0 + a.bias[n], z1 = v1 + a.bias[n + 1];
            if (a.z) *reinterpret_cast<float2*>(&a.z[m * a.cout + n]) = make_float2(z0, z1);
            if (a.sd)
              *reinterpret_cast<__nv_bfloat162*>(&a.sd[m * a.cout + n]) = __floats2bfloat162_rn(dsilu(z0), dsilu(z1));
            if (a.h)
              *reinterpret_cast<__nv_bfloat162*>(&a.h[m * a.cout + n]) = __floats2bfloat162_rn(silu(z0), silu(z1));
          } else if (n < N) {
            const float z0 = v0 + a.bias[n];
            if (a.z) a.z[m * a.cout + n] = z0;
            if (a.sd) a.sd[m * a.cout + n] = __float2bfloat16_rn(dsilu(z0));
            if (a.h) a.h[m * a.cout + n] = __float2bfloat16_rn(silu(z0));
          }
        } else if (MODE == MODE_BWD_DATA) {
          if (n + 1 < N) {
            float d0 = v0, d1 = v1;
            if (a.sdprev) {
              const float2 sp = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&a.sdprev[m * a.cin + n]));
              d0 *= sp.x;
              d1 *= sp.y;
            }
            *reinterpret_cast<__nv_bfloat162*>(&a.dzprev[m * a.cin + n]) = __floats2bfloat162_rn(d0, d1);
          } else if (n < N) {
            const float d0 = a.sdprev ? v0 * __bfloat162float(a.sdprev[m * a.cin + n]) : v0;
            a.dzprev[m * a.cin + n] = __float2bfloat16_rn(d0);
          }
        } else {
          if (n < N) atomicAdd(&a.dw[m * N + n], v0);
          if (n + 1 < N) atomicAdd(&a.dw[m * N + n + 1], v1);
        }
      }
}

// ---------------------------------------------------------------------------
// Tensor-core (tcgen05) convolution for forward and backward-data passes.
//
// One tile = 128 consecutive pixels of one image row (M = 128), all output
// channels (N = nout <= 256).  The CTA copies the tile's halo once: image rows
// y - d, y, y + d and columns x0 - d .. x0 + 127 + d, every gathered channel,
// zero outside the image, into shared memory in the no-swizzle K-major
// core-matrix layout
//     byte (kc * 3 * RW + r * RW + c) * 16 + 2 * (ci % 8),  kc = ci / 8, RW = 128 + 2d,
// i.e. the 16-byte channel chunk of halo pixel (r, c) in plane kc.  Pixels
// sit 16 bytes apart inside a plane, so the A operand of tap (dy, dx) is the
// same buffer with the descriptor's start moved by ((1 + sy) RW + d + sx d) * 16
// bytes ((sy, sx) = (dy, dx) forward, -(dy, dx) backward): nine taps, one
// copy.  The weights of all nine taps stay in shared memory for the whole
// persistent CTA in the same layout (rows = output channels).  One thread
// issues the 9 x (K / 16) tcgen05.mma.kind::f16 per tile into a TMEM
// accumulator (double-buffered: 2 x nout FP32 columns), tcgen05.commit
// signals an mbarrier, and the eight warps read the previous tile's
// accumulator with tcgen05.ld for the fused epilogue while the tensor core
// works on the current one.  Halo copies use cp.async (zero-fill) one tile
// ahead.  Every mbarrier wait is bounded; a wait that runs out sets *err,
// and the CTA stops, frees its TMEM and returns.
// ---------------------------------------------------------------------------
struct TcArgs {
  Geo g;
  int cg;              // gathered channels = K per tap (multiple of 16)
  int nout;            // output channels = N (multiple of 16, <= 256)
  int dil;
  const bf16* act;     // gathered activation, channels-last [P][cg]
  const bf16* wsrc;    // forward: W[nout][9][cg]; backward: WT[9][nout][cg]
  const float* bias;   // forward
  float* z;            // forward: the last layer's output [P][nout] (FP32), else nullptr
  bf16* h;             // forward: silu(z) (BF16), or nullptr
  bf16* sd;            // forward (training): silu'(z) (BF16), or nullptr
  const bf16* sdprev;  // backward: silu'(z) of the layer below [P][nout] (BF16), or nullptr
  bf16* dzprev;        // backward: output gradient [P][nout] (BF16)
  int* err;            // set to 1 when a wait runs out
  long long spin_limit;
};

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, long long limit) {
  const uint32_t addr = smem_u32(b);
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// shared-memory matrix descriptor: no swizzle, K-major, LBO = byte distance of
// K-adjacent core matrices, SBO = byte distance of M/N-adjacent core matrices
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;          // descriptor version for tcgen05
  return d;                        // base offset 0, layout type 0 (no swizzle)
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void tc_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Roles: warps 0-1 copy halos (cp.async, two tiles in flight, each thread
// waits for its own copies, fences them into the async proxy and arrives on
// the stage's "full" barrier); warp 2 (one lane) issues the MMAs of a tile
// once its halo is full and its accumulator empty, and commits to the
// stage's "empty" and the accumulator's "full" barriers; warps 3-10 drain an
// accumulator (warp w reads TMEM lane quarter w % 4 and half of the columns),
// release it and finish the epilogue.  Tile i uses halo stage and accumulator
// i & 1.
constexpr int kTcThreads = 352, kTcProducers = 64, kTcEpiWarps = 8;

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// bounded wait that also gives up once another role has aborted
__device__ __forceinline__ bool role_wait(uint64_t* b, uint32_t parity, long long limit, volatile int* abort_flag) {
  for (long long it = 0; it < limit; it += 64) {
    if (mbar_wait(b, parity, 64)) return true;
    if (*abort_flag) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
// 128-byte-swizzled descriptor (8-row atoms of 1024 bytes).  The swizzle
// phase follows the absolute shared-memory address (as TMA writes it), so a
// start moved by whole 128-byte rows inside an atom needs no base offset.
// lbo: K-major - unused inside one atom; MN-major - byte distance of the two
// 64-element halves of a 128-wide operand.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr, uint32_t lbo = 16) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;             // stride byte offset: next 8 rows
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;                       // SWIZZLE_128B
  return d;
}

// LAYOUT 0: no-swizzle core-matrix halo filled by cp.async (any cg that is a
// multiple of 16).  LAYOUT 1: cg = 64, halo rows of 128 bytes per pixel in the
// 128-byte-swizzled layout, filled by three TMA copies per tile (zero fill
// outside the image), weights stored in the same layout.
template <int MODE, int LAYOUT>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(const TcArgs a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  __shared__ __align__(8) uint64_t full_b[2], empty_b[2], accf_b[2], acce_b[2];
  __shared__ uint32_t tmem_slot;
  __shared__ float sbias[256];
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Geo& g = a.g;
  // 1024-aligned base (the swizzled layouts need it; the launch adds 1 KB of slack)
  uint8_t* tc_smem = tc_smem_raw + ((1024u - (smem_u32(tc_smem_raw) & 1023u)) & 1023u);
  const int d = a.dil, RW = LAYOUT ? (128 + 2 * d + 7) / 8 * 8 : 128 + 2 * d, planes = a.cg / 8, nout = a.nout;
  const uint32_t BSZ = 9u * a.cg * nout * 2, ASZ = LAYOUT ? 3u * RW * 128 : 6u * a.cg * RW, LBOA = 3u * RW * 16;
  const uint32_t ncols = nout * 2 <= 32 ? 32 : (nout * 2 <= 64 ? 64 : (nout * 2 <= 128 ? 128 : (nout * 2 <= 256 ? 256 : 512)));
  const int TX = (g.W + 127) / 128;
  const int64_t T = (int64_t)g.nb * g.H * TX;
  const int sgn = (MODE == MODE_FWD) ? 1 : -1;

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full_b[i], LAYOUT ? 1 : kTcProducers);
      mbar_init(&empty_b[i], 1);
      mbar_init(&accf_b[i], 1);
      mbar_init(&acce_b[i], kTcEpiWarps);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (MODE == MODE_FWD)
    for (int n = tid; n < nout; n += kTcThreads) sbias[n] = a.bias[n];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  // weights of the nine taps: chunk (t, kc, n) at ((t * planes + kc) * nout + n) * 16
  for (int e = tid; e < 9 * planes * nout; e += kTcThreads) {
    const int n = e % nout, kc = (e / nout) % planes, t = e / (nout * planes);
    const bf16* src = (MODE == MODE_FWD) ? a.wsrc + ((int64_t)n * 9 + t) * a.cg + 8 * kc
                                         : a.wsrc + ((int64_t)t * nout + n) * a.cg + 8 * kc;
    if (LAYOUT) cp16(tc_smem + (t * nout + n) * 128 + ((kc ^ (n & 7)) << 4), src, true);
    else cp16(tc_smem + ((t * planes + kc) * nout + n) * 16, src, true);
  }
  cp_commit();
  cp_wait<0>();
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool aborted = false;

  if (LAYOUT && warp < 2) {
    // ---------------- TMA producer (one lane) ----------------
    if (tid == 0) {
      int i = 0;
      for (int64_t tile = blockIdx.x; tile < T; tile += gridDim.x, ++i) {
        const int st = i & 1, k = i >> 1;
        if (k >= 1 && !role_wait(&empty_b[st], (k - 1) & 1, a.spin_limit, &abort_flag)) { aborted = true; break; }
        const int j = int(tile % TX);
        const int64_t rowid = tile / TX;
        const int y = int(rowid % g.H), img = int(rowid / g.H);
        mbar_expect_tx(&full_b[st], 3u * RW * 128);
        const uint32_t dst = smem_u32(tc_smem + BSZ + st * ASZ);
        for (int r = 0; r < 3; ++r)
          tma_load_4d(dst + r * RW * 128, &tmap, 0, 128 * j - d, y + (r - 1) * d, img, &full_b[st]);
      }
    }
    __syncwarp();
  } else if (warp < 2) {
    // ---------------- producers ----------------
    // chunk e = ptid + k * 64: plane kc = e % planes (fixed per thread), halo pixel q = e / planes
    const int ptid = tid, qstep = kTcProducers / planes, kc = ptid % planes;
    const int total_q = 3 * RW;
    int i = 0;
    for (int64_t tile = blockIdx.x; tile < T; tile += gridDim.x, ++i) {
      const int st = i & 1, k = i >> 1;
      if (k >= 1 && !role_wait(&empty_b[st], (k - 1) & 1, a.spin_limit, &abort_flag)) { aborted = true; break; }
      const int j = int(tile % TX);
      const int64_t rowid = tile / TX;
      const int y = int(rowid % g.H), x0 = 128 * j;
      uint8_t* dst0 = tc_smem + BSZ + st * ASZ + kc * LBOA;
      int q = ptid / planes, r = q / RW, c = q - r * RW;
      for (; q < total_q; q += qstep) {
        const int yy = y + (r - 1) * d, xx = x0 - d + c;
        const bool v = yy >= 0 && yy < g.H && xx >= 0 && xx < g.W;
        const bf16* src = v ? a.act + ((rowid + (int64_t)(r - 1) * d) * g.W + xx) * a.cg + 8 * kc : a.act;
        cp16(dst0 + (r * RW + c) * 16, src, v);
        c += qstep;
        while (c >= RW) { c -= RW; ++r; }
      }
      cp_commit();
      if (i >= 1) {
        cp_wait<1>();
        fence_proxy_async();
        mbar_arrive(&full_b[(i - 1) & 1]);
      }
    }
    cp_wait<0>();
    if (i >= 1 && !aborted) {
      fence_proxy_async();
      mbar_arrive(&full_b[(i - 1) & 1]);
    }
  } else if (warp == 2) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, nout);
      const uint32_t sm_base = smem_u32(tc_smem);
      int i = 0;
      for (int64_t tile = blockIdx.x; tile < T; tile += gridDim.x, ++i) {
        const int st = i & 1, k = i >> 1;
        if (!role_wait(&full_b[st], k & 1, a.spin_limit, &abort_flag)) { aborted = true; break; }
        if (k >= 1 && !role_wait(&acce_b[st], (k - 1) & 1, a.spin_limit, &abort_flag)) { aborted = true; break; }
        tc_fence_after();
        const uint32_t a0 = sm_base + BSZ + st * ASZ;
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const int sy = sgn * tap_dy(t), sx = sgn * tap_dx(t);
          if (LAYOUT) {
            // one descriptor per tap; the K slices step the 16-byte start-address field by 2 (32 bytes)
            const uint64_t ad0 = sdesc_sw128(a0 + (uint32_t)(((1 + sy) * RW + d + sx * d) * 128));
            const uint64_t bd0 = sdesc_sw128(sm_base + (uint32_t)(t * nout * 128));
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              tc_mma(tmem + (uint32_t)(st * nout), ad0 + 2u * kk, bd0 + 2u * kk, idesc, (t | kk) != 0);
          } else {
            const uint32_t aoff = a0 + (uint32_t)(((1 + sy) * RW + d + sx * d) * 16);
            const uint32_t boff = sm_base + (uint32_t)(t * planes * nout * 16);
            for (int kk = 0; kk < planes / 2; ++kk) {
              const uint64_t ad = sdesc(aoff + 2 * kk * LBOA, LBOA, 128);
              const uint64_t bd = sdesc(boff + 2 * kk * nout * 16, nout * 16, 128);
              tc_mma(tmem + (uint32_t)(st * nout), ad, bd, idesc, (t | kk) != 0);
            }
          }
        }
        tc_commit(&empty_b[st]);
        tc_commit(&accf_b[st]);
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    const int q4 = warp & 3, chalf = (warp - 3) >> 2;
    const int m = 32 * q4 + lane;
    const int cw = nout / 2;                     // columns of this warp: [chalf * cw, chalf * cw + cw)
    int i = 0;
    for (int64_t tile = blockIdx.x; tile < T; tile += gridDim.x, ++i) {
      const int b = i & 1, k = i >> 1;
      const bool ok_wait = role_wait(&accf_b[b], k & 1, a.spin_limit, &abort_flag);
      if (!__all_sync(0xffffffffu, ok_wait)) { aborted = true; break; }
      tc_fence_after();
      const int j = int(tile % TX);
      const int64_t rowid = tile / TX;
      const int x = 128 * j + m;
      const bool ok = x < g.W;
      const int64_t p = rowid * g.W + x;
      const int cend = chalf * cw + cw;
      int nc = 0;
      for (int c0 = chalf * cw; c0 < cend; c0 += nc) {
        float v[32];
        uint4 sdv[4];
        nc = cend - c0 >= 32 ? 32 : (cend - c0 >= 16 ? 16 : 8);
        if (MODE == MODE_BWD_DATA && a.sdprev && ok) {   // silu' of these columns, in flight during the TMEM load
          const uint4* src = reinterpret_cast<const uint4*>(a.sdprev + p * nout + c0);
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (8 * e < nc) sdv[e] = src[e];
        }
        const uint32_t ta = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(b * nout + c0);
        if (nc == 32) {
          tc_ld32(ta, v);
        } else {
          for (int e = 0; e < nc; e += 8) tc_ld8(ta + e, v + e);
        }
        if (c0 + nc >= cend) {   // the accumulator is in registers: release it to the MMA issuer
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acce_b[b]);
        }
        if (!ok) continue;
        for (int c1 = 0; c1 < nc; c1 += 8) {
          const int cc = c0 + c1;
          if (MODE == MODE_FWD) {
            float zz[8], sg[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              zz[e] = v[c1 + e] + sbias[cc + e];
              sg[e] = __fdividef(1.f, 1.f + __expf(-zz[e]));   // sigmoid, shared by silu and silu'
            }
            if (a.z) {
              float4* zd = reinterpret_cast<float4*>(a.z + p * nout + cc);
              zd[0] = make_float4(zz[0], zz[1], zz[2], zz[3]);
              zd[1] = make_float4(zz[4], zz[5], zz[6], zz[7]);
            }
            if (a.h) {
              __nv_bfloat162 hb[4];
#pragma unroll
              for (int e = 0; e < 4; ++e)
                hb[e] = __floats2bfloat162_rn(zz[2 * e] * sg[2 * e], zz[2 * e + 1] * sg[2 * e + 1]);
              *reinterpret_cast<uint4*>(a.h + p * nout + cc) = *reinterpret_cast<uint4*>(hb);
            }
            if (a.sd) {
              __nv_bfloat162 sb[4];
#pragma unroll
              for (int e = 0; e < 4; ++e)
                sb[e] = __floats2bfloat162_rn(sg[2 * e] * (1.f + zz[2 * e] * (1.f - sg[2 * e])),
                                              sg[2 * e + 1] * (1.f + zz[2 * e + 1] * (1.f - sg[2 * e + 1])));
              *reinterpret_cast<uint4*>(a.sd + p * nout + cc) = *reinterpret_cast<uint4*>(sb);
            }
          } else {
            float dd[8];
            if (a.sdprev) {
              const uint4 raw = sdv[c1 / 8];
              const __nv_bfloat162* sp = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(sp[e]);
                dd[2 * e] = v[c1 + 2 * e] * f.x;
                dd[2 * e + 1] = v[c1 + 2 * e + 1] * f.y;
              }
            } else {
#pragma unroll
              for (int e = 0; e < 8; ++e) dd[e] = v[c1 + e];
            }
            __nv_bfloat162 hb[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) hb[e] = __floats2bfloat162_rn(dd[2 * e], dd[2 * e + 1]);
            *reinterpret_cast<uint4*>(a.dzprev + p * nout + cc) = *reinterpret_cast<uint4*>(hb);
          }
        }
      }
    }
  }
  if (aborted) {
    abort_flag = 1;
    atomicOr(a.err, 1);
  }
  cp_wait<0>();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------
// Tensor-core weight gradient for 64-in / 64-out layers:
//     dW[co][t][ci] = sum_p dz[p][co] h[p + d o_t][ci].
// K = pixels, so both operands are MN-major in their natural channels-last
// layout: the halo of h (as in the forward kernel) and the tile's dz rows
// (one TMA box of 128 pixels x 64 channels), both 128-byte swizzled.  One MMA
// covers two taps: M = 128 rows = (tap t1: ci 0..63, tap t2: ci 0..63), the
// two halves being the two taps' shifted views of the halo (the descriptor's
// leading byte offset is their distance), N = 64 (co), K = 16 pixels.  Five
// tap pairs accumulate in TMEM (5 x 64 FP32 columns) over the CTA's run of
// tiles.  The last pair's second half reads a block of BF16 ones instead of a
// tap view, so its rows hold sum_p dz[p][co]: the bias gradient.  The CTA
// then writes its partial sums (weights, then bias), and k_sum_parts adds the
// CTAs' parts in a fixed order.
// ---------------------------------------------------------------------------
struct WgArgs {
  Geo g;
  int dil;
  float* part;          // [gridDim.x][64 * 9 * 64 + 64]: weight part, then bias part
  int* err;
  long long spin_limit;
};
constexpr int kWgThreads = 128, kWgMaxParts = 160;
constexpr size_t kWgSmem = 220 * 1024;    // two stages of halo + dz tile, the ones block, alignment: <= 173 KB
constexpr uint32_t kWgDz = 128 * 128;     // one dz tile: 128 pixels x 128 bytes
constexpr int64_t kWgPart = 64 * 9 * 64 + 64;

__global__ void __launch_bounds__(kWgThreads, 1) k_wgrad_tc(const WgArgs a, const __grid_constant__ CUtensorMap tm_h,
                                                            const __grid_constant__ CUtensorMap tm_dz) {
  extern __shared__ __align__(1024) uint8_t wg_smem_raw[];
  __shared__ __align__(8) uint64_t full_b[2], empty_b[2], done_b;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  uint8_t* sm = wg_smem_raw + ((1024u - (smem_u32(wg_smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Geo& g = a.g;
  const int d = a.dil, RW = (128 + 2 * d + 7) / 8 * 8;
  const uint32_t HALO = 3u * RW * 128, STG = HALO + kWgDz;
  const int TX = (g.W + 127) / 128;
  const int64_t T = (int64_t)g.nb * g.H * TX;
  const int64_t t_begin = T * blockIdx.x / gridDim.x, t_end = T * (blockIdx.x + 1) / gridDim.x;
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full_b[i], 1);
      mbar_init(&empty_b[i], 1);
    }
    mbar_init(&done_b, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  // the ones block (16 KB of BF16 1.0) after the two stages
  {
    uint4* ones = reinterpret_cast<uint4*>(sm + 2 * STG);
    const uint32_t one2 = 0x3F803F80u;
    for (int i = tid; i < (int)(kWgDz / 16); i += kWgThreads) ones[i] = make_uint4(one2, one2, one2, one2);
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool aborted = false;
  const int64_t ntiles = t_end - t_begin;

  if (warp == 0) {
    if (lane == 0) {   // producer
      for (int64_t i = 0; i < ntiles; ++i) {
        const int st = int(i & 1);
        const int64_t k = i >> 1;
        if (k >= 1 && !role_wait(&empty_b[st], (uint32_t)((k - 1) & 1), a.spin_limit, &abort_flag)) {
          aborted = true;
          break;
        }
        const int64_t tile = t_begin + i;
        const int j = int(tile % TX);
        const int64_t rowid = tile / TX;
        const int y = int(rowid % g.H), img = int(rowid / g.H);
        mbar_expect_tx(&full_b[st], STG);
        const uint32_t dst = smem_u32(sm + st * STG);
        for (int r = 0; r < 3; ++r)
          tma_load_4d(dst + r * RW * 128, &tm_h, 0, 128 * j - d, y + (r - 1) * d, img, &full_b[st]);
        tma_load_4d(dst + HALO, &tm_dz, 0, 128 * j, y, img, &full_b[st]);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      const uint32_t idesc = idesc_bf16(128, 64) | (1u << 15) | (1u << 16);   // A and B MN-major
      const uint32_t base = smem_u32(sm);
      for (int64_t i = 0; i < ntiles; ++i) {
        const int st = int(i & 1);
        if (!role_wait(&full_b[st], (uint32_t)((i >> 1) & 1), a.spin_limit, &abort_flag)) {
          aborted = true;
          break;
        }
        tc_fence_after();
        const uint32_t halo = base + st * STG, dzt = halo + HALO;
#pragma unroll
        for (int pi = 0; pi < 5; ++pi) {
          const int t1 = 2 * pi, t2 = 2 * pi + 1;
          const uint32_t v1 = halo + (uint32_t)(((1 + tap_dy(t1)) * RW + d + tap_dx(t1) * d) * 128);
          const uint32_t v2 = pi < 4 ? halo + (uint32_t)(((1 + tap_dy(t2)) * RW + d + tap_dx(t2) * d) * 128)
                                     : base + 2 * STG;   // ones: the bias gradient
          // K steps of 16 pixels move both starts by 2048 bytes: 128 in the 16-byte address field
          const uint64_t ad0 = sdesc_sw128(v1, v2 - v1), bd0 = sdesc_sw128(dzt);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk)
            tc_mma(tmem + (uint32_t)(pi * 64), ad0 + 128u * kk, bd0 + 128u * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
        }
        tc_commit(&empty_b[st]);
      }
      if (!aborted) tc_commit(&done_b);
    }
    __syncwarp();
  }
  // all four warps: drain the accumulators into this CTA's part
  if (__syncthreads_or(aborted)) aborted = true;
  if (!aborted && ntiles > 0) {
    const bool ok = role_wait(&done_b, 0, a.spin_limit, &abort_flag);
    if (__syncthreads_or(!ok)) aborted = true;
  }
  if (!aborted) {
    tc_fence_after();
    float* part = a.part + (int64_t)blockIdx.x * kWgPart;
    const int r = 32 * warp + lane;          // accumulator row = (tap half, ci)
    for (int pi = 0; pi < 5; ++pi) {
      float v[64];
      if (ntiles > 0) {
        tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(pi * 64), v);
        tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(pi * 64 + 32), v + 32);
      } else {
        for (int c = 0; c < 64; ++c) v[c] = 0.f;
      }
      const int t = 2 * pi + (r >> 6), ci = r & 63;
      if (t < 9)
        for (int co = 0; co < 64; ++co) part[((int64_t)co * 9 + t) * 64 + ci] = v[co];
      else if (r == 64)
        for (int co = 0; co < 64; ++co) part[64 * 9 * 64 + co] = v[co];
    }
  }
  if (aborted) {
    abort_flag = 1;
    if (tid == 0) atomicOr(a.err, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512));
}

// dw[i] += sum over the parts (fixed order) for the weights, db[c] likewise for the bias
__global__ void k_sum_parts(const float* __restrict__ part, int nparts, float* __restrict__ dw,
                            float* __restrict__ db) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < kWgPart; i += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int b = 0; b < nparts; ++b) acc += part[(int64_t)b * kWgPart + i];
    if (i < 64 * 9 * 64) dw[i] += acc;
    else db[i - 64 * 9 * 64] += acc;
  }
}

// WT[t][ci][co] = W[co][t][ci] (BF16), the backward-data operand layout
__global__ void k_transpose_w(const bf16* __restrict__ w, bf16* __restrict__ wt, int cin, int cout) {
  const int64_t n = (int64_t)cout * 9 * cin;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int ci = int(i % cin), t = int((i / cin) % 9), co = int(i / (9 * (int64_t)cin));
    wt[((int64_t)t * cin + ci) * cout + co] = w[i];
  }
}

// Per-state sums of |psi_in|^2 and |psi_out|^2 (FP64): grid (kMassBlocks, nb), 256 threads;
// partial sums to part[(n * kMassBlocks + block) * 2 + {0, 1}].
constexpr int kMassBlocks = 32;
__global__ void k_state_mass(const float2* __restrict__ in, const float2* __restrict__ out, int64_t HW,
                             double* __restrict__ part) {
  __shared__ double r0[256], r1[256];
  const int64_t base = (int64_t)blockIdx.y * HW;
  double a = 0.0, b = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += (int64_t)gridDim.x * blockDim.x) {
    const float2 u = in[base + p], v = out[base + p];
    a += double(u.x) * u.x + double(u.y) * u.y;
    b += double(v.x) * v.x + double(v.y) * v.y;
  }
  r0[threadIdx.x] = a;
  r1[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      r0[threadIdx.x] += r0[threadIdx.x + o];
      r1[threadIdx.x] += r1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[((int64_t)blockIdx.y * kMassBlocks + blockIdx.x) * 2] = r0[0];
    part[((int64_t)blockIdx.y * kMassBlocks + blockIdx.x) * 2 + 1] = r1[0];
  }
}

// Per-state sums of |psi + y|^2 (the network's raw output, y with a pc-channel row stride) and
// |target|^2, in the layout of k_state_mass.
__global__ void k_state_mass_res(const float2* __restrict__ psi, const float* __restrict__ y, int pc,
                                 const float2* __restrict__ target, int64_t HW, double* __restrict__ part) {
  __shared__ double r0[256], r1[256];
  const int64_t base = (int64_t)blockIdx.y * HW;
  double a = 0.0, b = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += (int64_t)gridDim.x * blockDim.x) {
    const float2 u = psi[base + p], t = target[base + p];
    const float2 d = *reinterpret_cast<const float2*>(y + (base + p) * pc);
    const float ox = u.x + d.x, oy = u.y + d.y;
    a += double(ox) * ox + double(oy) * oy;
    b += double(t.x) * t.x + double(t.y) * t.y;
  }
  r0[threadIdx.x] = a;
  r1[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      r0[threadIdx.x] += r0[threadIdx.x + o];
      r1[threadIdx.x] += r1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[((int64_t)blockIdx.y * kMassBlocks + blockIdx.x) * 2] = r0[0];
    part[((int64_t)blockIdx.y * kMassBlocks + blockIdx.x) * 2 + 1] = r1[0];
  }
}

// Per-state sums of |a - b|^2 and |b|^2, in the layout of k_state_mass.
__global__ void k_state_diff(const float2* __restrict__ a_, const float2* __restrict__ b_, int64_t HW,
                             double* __restrict__ part) {
  __shared__ double r0[256], r1[256];
  const int64_t base = (int64_t)blockIdx.y * HW;
  double a = 0.0, b = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += (int64_t)gridDim.x * blockDim.x) {
    const float2 u = a_[base + p], v = b_[base + p];
    const double dx = double(u.x) - v.x, dy = double(u.y) - v.y;
    a += dx * dx + dy * dy;
    b += double(v.x) * v.x + double(v.y) * v.y;
  }
  r0[threadIdx.x] = a;
  r1[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      r0[threadIdx.x] += r0[threadIdx.x + o];
      r1[threadIdx.x] += r1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[((int64_t)blockIdx.y * kMassBlocks + blockIdx.x) * 2] = r0[0];
    part[((int64_t)blockIdx.y * kMassBlocks + blockIdx.x) * 2 + 1] = r1[0];
  }
}

// out2[2b], out2[2b + 1]: the two per-state sums, partials added in a fixed order (one thread per state)
__global__ void k_state_sums(const double* __restrict__ part, int nb, double* __restrict__ out2) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double a = 0.0, c = 0.0;
  for (int i = 0; i < kMassBlocks; ++i) {
    a += part[((int64_t)b * kMassBlocks + i) * 2];
    c += part[((int64_t)b * kMassBlocks + i) * 2 + 1];
  }
  out2[2 * b] = a;
  out2[2 * b + 1] = c;
}

// The mass term of the loss, mu mean_b delta_b^2 with delta_b = (M_out - M_t) / M_t: per state the
// coefficient of its gradient, d/d out = coef_b out with coef_b = 4 mu delta_b / (nb M_t), and the
// term itself into *loss (one thread per state).
__global__ void k_mass_coef(const double* __restrict__ part, int nb, double mu, double* __restrict__ coef,
                            double* __restrict__ loss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double mo = 0.0, mt = 0.0;
  for (int i = 0; i < kMassBlocks; ++i) {
    mo += part[((int64_t)b * kMassBlocks + i) * 2];
    mt += part[((int64_t)b * kMassBlocks + i) * 2 + 1];
  }
  const double delta = mt > 0.0 ? (mo - mt) / mt : 0.0;
  coef[b] = mt > 0.0 ? 4.0 * mu * delta / (double(nb) * mt) : 0.0;
  atomicAdd(loss, mu * delta * delta / double(nb));
}

// out *= sqrt(M_in / M_out) per state (same grid as k_state_mass; partials summed in a fixed order)
__global__ void k_project(float2* __restrict__ out, int64_t HW, const double* __restrict__ part) {
  __shared__ float r;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < kMassBlocks; ++i) {
      a += part[((int64_t)blockIdx.y * kMassBlocks + i) * 2];
      b += part[((int64_t)blockIdx.y * kMassBlocks + i) * 2 + 1];
    }
    r = b > 0.0 ? float(sqrt(a / b)) : 1.f;
  }
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.y * HW;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = out[base + p];
    out[base + p] = make_float2(v.x * r, v.y * r);
  }
}

// The two-channel ends of the network run as pc-channel layers (pc = C when C
// is 16, 32, 48 or 64, else 16): the input activation carries (Re, Im, 0 ...),
// the last layer computes pc outputs of which channels 2.. have zero weights
// and bias, and its output gradient is written with the same pc stride.
// Every layer then fits the same kernels as the inner ones; the padding adds
// exact zeros only.
__host__ __device__ inline int pad_width(int C) { return (C % 16 == 0 && C <= 64) ? C : 16; }

// Input features per pixel: Re psi, Im psi, |psi|^2 Re psi, |psi|^2 Im psi
// (the last two are the cubic term of the NLSE, so that one Euler step of
// F(psi) is linear in the features).  Each feature x enters the first layer
// as two BF16 channels, x_hi = bf16(x) and x_lo = bf16(x - x_hi), multiplied
// by the same weight (the padded copy repeats W_0 for both), so the first
// convolution sees the features at about 16 significant bits instead of 8.
constexpr int kIn = 4;

// complex state -> pc-channel BF16 input (the kIn features, zeros); one thread per 16-byte chunk
__global__ void k_pack_input(const float2* __restrict__ psi, int64_t P, int pc, bf16* __restrict__ h) {
  const int cpp = pc / 8;
  uint4* dst = reinterpret_cast<uint4*>(h);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P * cpp; q += (int64_t)gridDim.x * blockDim.x) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (q % cpp == 0) {   // channels 0..3: hi parts, 4..7: lo parts of the kIn features
      const float2 z = psi[q / cpp];
      const float r = fmaf(z.x, z.x, z.y * z.y);
      const float f[4] = {z.x, z.y, r * z.x, r * z.y};
      float hi[4], lo[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        hi[e] = __bfloat162float(__float2bfloat16_rn(f[e]));
        lo[e] = f[e] - hi[e];
      }
      const __nv_bfloat162 a0 = __floats2bfloat162_rn(hi[0], hi[1]), a1 = __floats2bfloat162_rn(hi[2], hi[3]);
      const __nv_bfloat162 b0 = __floats2bfloat162_rn(lo[0], lo[1]), b1 = __floats2bfloat162_rn(lo[2], lo[3]);
      v.x = *reinterpret_cast<const uint32_t*>(&a0);
      v.y = *reinterpret_cast<const uint32_t*>(&a1);
      v.z = *reinterpret_cast<const uint32_t*>(&b0);
      v.w = *reinterpret_cast<const uint32_t*>(&b1);
    }
    dst[q] = v;
  }
}

// Per-state max |psi| partials: grid (kMassBlocks, nb), 256 threads -> part[n * kMassBlocks + block]
__global__ void k_state_amax(const float2* __restrict__ psi, int64_t HW, float* __restrict__ part) {
  __shared__ float r[256];
  const int64_t base = (int64_t)blockIdx.y * HW;
  float m = 0.f;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = psi[base + p];
    m = fmaxf(m, fmaf(v.x, v.x, v.y * v.y));
  }
  r[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) r[threadIdx.x] = fmaxf(r[threadIdx.x], r[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)blockIdx.y * kMassBlocks + blockIdx.x] = sqrtf(r[0]);
}

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Training input with noise: out = psi + sigma * max|psi_n| * (g_re + i g_im), g standard normal
// (Box-Muller on two SplitMix64 uniforms per component, counter = seed-mixed element index).
__global__ void k_add_noise(const float2* __restrict__ psi, int64_t HW, int nb, const float* __restrict__ amax_part,
                            float sigma, uint64_t seed, float2* __restrict__ out) {
  __shared__ float amp;
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int i = 0; i < kMassBlocks; ++i) m = fmaxf(m, amax_part[(int64_t)blockIdx.y * kMassBlocks + i]);
    amp = sigma * m;
  }
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.y * HW;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t c = (uint64_t)(base + p) * 4u;
    float g[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float u1 = (float)((splitmix64(seed ^ (c + 2 * e)) >> 40) + 1) * (1.f / 16777217.f);   // (0, 1]
      const float u2 = (float)(splitmix64(seed ^ (c + 2 * e + 1)) >> 40) * (1.f / 16777216.f);      // [0, 1)
      g[e] = sqrtf(-2.f * logf(u1)) * cosf(6.283185307f * u2);
    }
    const float2 v = psi[base + p];
    out[base + p] = make_float2(v.x + amp * g[0], v.y + amp * g[1]);
  }
}

// psi_out = psi_in + (y_0 + i y_1), y with a pc-channel row stride
__global__ void k_residual(const float2* __restrict__ psi, const float* __restrict__ y, int64_t P, int pc,
                           float2* __restrict__ out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = psi[p];
    const float2 d = *reinterpret_cast<const float2*>(y + p * pc);
    out[p] = make_float2(v.x + d.x, v.y + d.y);
  }
}

// MSE loss (FP64 partial sums) and its gradient w.r.t. y, written as the BF16
// output gradient of the last layer (pc-channel rows, channels 2.. zero); one
// thread per 16-byte chunk of that gradient
// With coef (the mass term, k_mass_coef), coef[p / HW] psi_out[p] is added to the gradient.
__global__ void k_mse(const float2* __restrict__ psi, const float* __restrict__ y, const float2* __restrict__ target,
                      int64_t P, int pc, bf16* __restrict__ dz, double* __restrict__ loss_acc,
                      const double* __restrict__ coef, int64_t HW) {
  __shared__ double red[256];
  double s = 0.0;
  const float scale = 2.f / float(2 * P);
  const int cpp = pc / 8;
  uint4* dst = reinterpret_cast<uint4*>(dz);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P * cpp; q += (int64_t)gridDim.x * blockDim.x) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (q % cpp == 0) {
      const int64_t p = q / cpp;
      const float2 u = psi[p], t = target[p];
      const float2 d = *reinterpret_cast<const float2*>(y + p * pc);
      const float ex = u.x + d.x - t.x, ey = u.y + d.y - t.y;
      s += double(ex) * ex + double(ey) * ey;
      float gx = scale * ex, gy = scale * ey;
      if (coef) {
        const float cb = float(coef[p / HW]);
        gx = fmaf(cb, u.x + d.x, gx);
        gy = fmaf(cb, u.y + d.y, gy);
      }
      const __nv_bfloat162 g = __floats2bfloat162_rn(gx, gy);
      v.x = *reinterpret_cast<const uint32_t*>(&g);
    }
    dst[q] = v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss_acc, red[0] / double(2 * P));
}

// db[c] += sum over pixels of dz[p * stride + c] for c < creal (stride <= 256;
// 256 threads: thread t takes channel t % stride of every (256 / stride)-th pixel)
__global__ void k_bias_grad(const bf16* __restrict__ dz, int64_t P, int stride, int creal, float* __restrict__ db) {
  __shared__ float red[256];
  const int groups = 256 / stride, c = threadIdx.x % stride, gi = threadIdx.x / stride;
  float s = 0.f;
  if (gi < groups)
    for (int64_t p = (int64_t)blockIdx.x * groups + gi; p < P; p += (int64_t)gridDim.x * groups)
      s += __bfloat162float(dz[p * stride + c]);
  red[threadIdx.x] = s;
  __syncthreads();
  if ((int)threadIdx.x < stride) {
    float t = 0.f;
    for (int g = 0; g < groups; ++g) t += red[g * stride + threadIdx.x];
    if ((int)threadIdx.x < creal) atomicAdd(&db[threadIdx.x], t);
  }
}

// Padded operand copies of the end layers (BF16 weights from the BF16 copy, FP32 bias):
//   w0[co][t][c]   = W_0[co][t][c % kIn] for c < 2 kIn, else 0  (C x 9 x pc; hi and lo channels)
//   wl[o][t][ci]   = W_{L-1}[o][t][ci] for o < 2, else 0        (pc x 9 x C)
//   wlt[t][ci][o]  = the same, transposed for backward-data     (9 x C x pc)
//   bl[o]          = b_{L-1}[o] for o < 2, else 0
__global__ void k_pad_ends(const bf16* __restrict__ w0src, const bf16* __restrict__ wlsrc,
                           const float* __restrict__ blsrc, int C, int pc, bf16* __restrict__ w0,
                           bf16* __restrict__ wl, bf16* __restrict__ wlt, float* __restrict__ bl) {
  const bf16 zero = __float2bfloat16_rn(0.f);
  const int64_t n = (int64_t)C * 9 * pc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    {   // w0, i = (co * 9 + t) * pc + c
      const int c = int(i % pc);
      const int64_t ct = i / pc;
      w0[i] = c < 2 * kIn ? w0src[ct * kIn + (c % kIn)] : zero;
    }
    {   // wl, i = (o * 9 + t) * C + ci
      const int64_t o = i / (9 * (int64_t)C);
      wl[i] = o < 2 ? wlsrc[i] : zero;
    }
    {   // wlt, i = (t * C + ci) * pc + o
      const int o = int(i % pc);
      const int64_t tc = i / pc;
      const int ci = int(tc % C), t = int(tc / C);
      wlt[i] = o < 2 ? wlsrc[((int64_t)o * 9 + t) * C + ci] : zero;
    }
    if (i < pc) bl[i] = i < 2 ? blsrc[i] : 0.f;
  }
}

// grad += the real part of a padded layer's gradient (scratch: weights, then pc bias slots):
//   first layer: W[(co * 9 + t) * kIn + c] += scr[.. * pc + c] + scr[.. * pc + kIn + c] (hi + lo); b[co] += scr[nw + co]
//   last layer:  W[i] += scr[i] for i < 2 * 9 * C (rows 0, 1);             b[o] += scr[nw + o], o < 2
__global__ void k_unpad_grad(const float* __restrict__ scr, float* __restrict__ dw, float* __restrict__ db, int C,
                             int pc, int first) {
  const int64_t nw = (int64_t)C * 9 * pc, n = (int64_t)9 * C * (first ? kIn : 2);
  const int nb = first ? C : 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n + nb; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n)
      dw[i] += first ? scr[(i / kIn) * pc + (i % kIn)] + scr[(i / kIn) * pc + kIn + (i % kIn)] : scr[i];
    else db[i - n] += scr[nw + (i - n)];
  }
}

// Adam step on the FP32 masters, refreshing the BF16 copies
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m, float* __restrict__ v,
                       bf16* __restrict__ pb, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * g, vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = w;
    pb[i] = __float2bfloat16_rn(w);
  }
}

__global__ void k_to_bf16(const float* __restrict__ p, bf16* __restrict__ pb, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    pb[i] = __float2bfloat16_rn(p[i]);
}

// SplitMix64-based uniform in [-1, 1) for parameter initialisation (counter-based, seeded)
__global__ void k_init(float* __restrict__ p, int64_t off, int64_t n, float scale, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)(off + i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = double(z >> 11) * (1.0 / 9007199254740992.0);
    p[off + i] = scale * float(2.0 * u - 1.0);
  }
}

int grid1d(int64_t n) {
  int64_t b = (n + 255) / 256;
  return int(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

}  // namespace

struct nlse_sur {
  int H, W, C, L, max_batch;
  int dil[kMaxLayers];
  float* params;                  // caller-owned FP32 masters
  int64_t nparam;
  std::vector<int64_t> w_off, b_off;   // offsets of W_l and b_l in params
  cudaStream_t stream;
  // workspace carve
  bf16* pbf;                      // BF16 copy of params
  bf16* pbfT;                     // BF16 transposed weights WT[t][ci][co] per layer (at the same offsets)
  float* grad;                    // FP32 gradients (param layout)
  float* m1;
  float* m2;
  double* loss;
  double* mass_part;              // [max_batch][kMassBlocks][2]
  double* mstat;                  // [2 max_batch]: the mass term's gradient coefficients, or per-state sum pairs
  double mass_weight;             // weight of the mass term in the loss (0: plain MSE)
  float* amax_part;               // [max_batch][kMassBlocks]
  float2* xnoisy;                 // noisy training input [max_batch][H][W]
  uint64_t seed;
  int pc;                         // padded width of the two-channel ends
  bf16* hin;                      // input activation, pc channels (Re, Im, zeros)
  bf16* pw0;                      // padded first-layer weights [C][9][pc]
  bf16* pwL;                      // padded last-layer weights [pc][9][C]
  bf16* pwLT;                     // its backward-data layout [9][C][pc]
  float* pbL;                     // padded last-layer bias [pc]
  float* wscr;                    // padded-layer gradient scratch [C * 9 * pc] weights + [pc] bias
  float* wgpart;                  // per-CTA weight-gradient parts of the tensor-core kernel (C = 64 only)
  float* y;                       // last layer's output, pc-channel rows (FP32)
  std::vector<bf16*> sd;          // silu'(z) of layers 0..L-2 (BF16; training)
  std::vector<bf16*> h;           // activations, layer 0..L-2
  int* err;                       // device flag: a bounded wait in a tensor-core kernel ran out
  int num_sms;
  int use_tc;                     // tcgen05 kernels for eligible forward / backward-data layers
  bf16* dzA;                      // gradient ping-pong buffers (max(C, pc) channels)
  bf16* dzB;
  int64_t adam_t;
};

namespace {

int cin_of(const nlse_sur* s, int l) { return l == 0 ? kIn : s->C; }
int cout_of(const nlse_sur* s, int l) { return l == s->L - 1 ? 2 : s->C; }

int64_t param_count(int C, int L) {
  int64_t n = 0;
  for (int l = 0; l < L; ++l) {
    const int ci = l == 0 ? kIn : C, co = l == L - 1 ? 2 : C;
    n += (int64_t)co * 9 * ci + co;
  }
  return n;
}

size_t ws_bytes(int H, int W, int C, int L, int max_batch) {
  const int64_t P = (int64_t)max_batch * H * W, np = param_count(C, L);
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t off = 0;
  off = al(off + np * 2);            // pbf
  off = al(off + np * 2);            // pbfT
  off = al(off + np * 4) * 1;        // grad
  off = al(off + np * 4);            // m1
  off = al(off + np * 4);            // m2
  off = al(off + 64);                // loss
  off = al(off + (size_t)max_batch * kMassBlocks * 2 * 8);   // mass_part
  off = al(off + (size_t)max_batch * 2 * 8);                  // mstat
  off = al(off + (size_t)max_batch * kMassBlocks * 4);       // amax_part
  off = al(off + P * 8);                                      // xnoisy
  off = al(off + 16);                // err
  const int pc = pad_width(C);
  off = al(off + P * pc * 2);        // hin
  off = al(off + (size_t)C * 9 * pc * 2);     // pw0
  off = al(off + (size_t)C * 9 * pc * 2);     // pwL
  off = al(off + (size_t)C * 9 * pc * 2);     // pwLT
  off = al(off + pc * 4);                     // pbL
  off = al(off + ((size_t)C * 9 * pc + pc) * 4);   // wscr
  off = al(off + (C == 64 ? (size_t)kWgMaxParts * kWgPart * 4 : 0));   // wgpart
  off = al(off + P * pc * 4);                                   // y
  for (int l = 0; l < L - 1; ++l) off = al(off + P * C * 2);    // sd
  for (int l = 0; l < L - 1; ++l) off = al(off + P * C * 2);    // h
  const int64_t cz = C > pc ? C : pc;
  off = al(off + P * cz * 2);        // dzA
  off = al(off + P * cz * 2);        // dzB
  return off;
}

// layout 1 (TMA, 128-byte swizzle) serves 64 gathered channels; layout 0 the rest
int tc_layout(int cg) { return cg == 64 ? 1 : 0; }

size_t tc_smem_bytes(int cg, int nout, int dil) {
  const size_t halo = tc_layout(cg) ? (size_t)3 * ((128 + 2 * dil + 7) / 8 * 8) * 128
                                    : (size_t)6 * cg * (128 + 2 * dil);
  return (size_t)9 * cg * nout * 2 + 2 * halo + 1024;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 4D map over a channels-last BF16 activation [nb][H][W][64]: box of 64
// channels x rw pixels of one row, 128-byte swizzle, zero fill outside.
bool halo_tmap(CUtensorMap* m, const bf16* act, int nb, int H, int W, int rw) {
  EncodeTiledFn fn = reinterpret_cast<EncodeTiledFn>(nlse::tensor_map_encoder());
  if (!fn) return false;
  const cuuint64_t dims[4] = {64, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)nb};
  const cuuint64_t strides[3] = {128, (cuuint64_t)W * 128, (cuuint64_t)H * W * 128};
  const cuuint32_t box[4] = {64, (cuuint32_t)rw, 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(act), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// gathered channels: a multiple of 16 whose 8-channel planes divide the 64 copying threads
bool tc_ok(int cg, int nout, int dil) {
  return cg % 16 == 0 && kTcProducers % (cg / 8) == 0 && nout % 16 == 0 && nout >= 16 && nout <= 256 &&
         dil <= 16 && tc_smem_bytes(cg, nout, dil) <= 220 * 1024;
}

bool fast_ok(int mode, int cin, int cout) {
  if (mode == MODE_FWD) return cin % 8 == 0 && cout % 2 == 0;
  if (mode == MODE_BWD_DATA) return cout % 8 == 0 && cin % 2 == 0;
  return cout % 8 == 0 && cin % 8 == 0;
}

// Operands of layer l as the kernels see them (the end layers padded to 16 channels).
struct LayerOps {
  int cin, cout;
  const bf16* w;
  const bf16* wt;
  const float* bias;
  float* dw;
  float* db;
};
LayerOps layer_ops(const nlse_sur* s, int l) {
  const bool first = l == 0, last = l == s->L - 1;
  LayerOps o;
  o.cin = first ? s->pc : s->C;
  o.cout = last ? s->pc : s->C;
  o.w = first ? s->pw0 : (last ? s->pwL : s->pbf + s->w_off[l]);
  o.wt = last ? s->pwLT : s->pbfT + s->w_off[l];
  o.bias = last ? s->pbL : s->params + s->b_off[l];
  o.dw = (first || last) ? s->wscr : s->grad + s->w_off[l];
  o.db = (first || last) ? s->wscr + (int64_t)s->C * 9 * s->pc : s->grad + s->b_off[l];
  return o;
}

// Returns through *bias_done whether the weight-gradient kernel also produced the bias gradient.
cudaError_t conv(const nlse_sur* s, int mode, int l, int nb, const bf16* x, const bf16* dz, float* z, bf16* h,
                 bf16* sd, const bf16* sdprev, bf16* dzprev, bool* bias_done = nullptr) {
  if (bias_done) *bias_done = false;
  const LayerOps o = layer_ops(s, l);
  ConvArgs a;
  memset(&a, 0, sizeof(a));
  a.g = {nb, s->H, s->W};
  a.cin = o.cin;
  a.cout = o.cout;
  a.dil = s->dil[l];
  a.x = x;
  a.dz = dz;
  a.w = o.w;
  a.bias = o.bias;
  a.z = z;
  a.h = h;
  a.sd = sd;
  a.sdprev = sdprev;
  a.dzprev = dzprev;
  a.dw = o.dw;
  const int64_t P = (int64_t)nb * s->H * s->W;
  const bf16* wt = o.wt;
  if (s->use_tc && mode != MODE_WGRAD) {
    const int cg = mode == MODE_FWD ? a.cin : a.cout, nout = mode == MODE_FWD ? a.cout : a.cin;
    if (tc_ok(cg, nout, a.dil)) {
      TcArgs t;
      memset(&t, 0, sizeof(t));
      t.g = a.g;
      t.cg = cg;
      t.nout = nout;
      t.dil = a.dil;
      t.act = mode == MODE_FWD ? x : dz;
      t.wsrc = mode == MODE_FWD ? a.w : wt;
      t.bias = a.bias;
      t.z = z;
      t.h = h;
      t.sd = sd;
      t.sdprev = sdprev;
      t.dzprev = dzprev;
      t.err = s->err;
      t.spin_limit = 1ll << 24;
      const int64_t tiles = (int64_t)nb * s->H * ((s->W + 127) / 128);
      const size_t smem = tc_smem_bytes(cg, nout, a.dil);
      const int64_t per_sm = smem <= 100 * 1024 ? 2 : 1;
      const unsigned grid = (unsigned)(tiles < s->num_sms * per_sm ? tiles : s->num_sms * per_sm);
      CUtensorMap tm;
      memset(&tm, 0, sizeof(tm));
      if (tc_layout(cg)) {
        if (!halo_tmap(&tm, t.act, nb, s->H, s->W, (128 + 2 * a.dil + 7) / 8 * 8)) return cudaErrorInvalidValue;
        if (mode == MODE_FWD) k_conv_tc<MODE_FWD, 1><<<grid, kTcThreads, smem, s->stream>>>(t, tm);
        else k_conv_tc<MODE_BWD_DATA, 1><<<grid, kTcThreads, smem, s->stream>>>(t, tm);
      } else {
        if (mode == MODE_FWD) k_conv_tc<MODE_FWD, 0><<<grid, kTcThreads, smem, s->stream>>>(t, tm);
        else k_conv_tc<MODE_BWD_DATA, 0><<<grid, kTcThreads, smem, s->stream>>>(t, tm);
      }
      return cudaGetLastError();
    }
  }
  if (s->use_tc && mode == MODE_WGRAD && a.cin == 64 && a.cout == 64 && a.dil <= 16) {
    const int rw = (128 + 2 * a.dil + 7) / 8 * 8;
    CUtensorMap th, tz;
    if (!halo_tmap(&th, x, nb, s->H, s->W, rw) || !halo_tmap(&tz, dz, nb, s->H, s->W, 128))
      return cudaErrorInvalidValue;
    WgArgs w;
    memset(&w, 0, sizeof(w));
    w.g = a.g;
    w.dil = a.dil;
    w.part = s->wgpart;
    w.err = s->err;
    w.spin_limit = 1ll << 24;
    const int grid = s->num_sms < kWgMaxParts ? s->num_sms : kWgMaxParts;
    k_wgrad_tc<<<grid, kWgThreads, kWgSmem, s->stream>>>(w, th, tz);
    k_sum_parts<<<grid1d(kWgPart), 256, 0, s->stream>>>(s->wgpart, grid, a.dw, layer_ops(s, l).db);
    if (bias_done) *bias_done = true;
    return cudaGetLastError();
  }
  if (fast_ok(mode, a.cin, a.cout)) {
    if (mode == MODE_FWD) {
      dim3 grid((unsigned)((P + 127) / 128), (unsigned)((a.cout + 63) / 64));
      k_conv_fast<MODE_FWD, 4, 2><<<grid, 256, 0, s->stream>>>(a, wt);
    } else if (mode == MODE_BWD_DATA) {
      dim3 grid((unsigned)((P + 127) / 128), (unsigned)((a.cin + 63) / 64));
      k_conv_fast<MODE_BWD_DATA, 4, 2><<<grid, 256, 0, s->stream>>>(a, wt);
    } else {
      // split the pixel (K) range so that the grid holds about four CTAs per SM
      const int64_t gx = (a.cout + 63) / 64, gy = (9 * a.cin + 127) / 128;
      int64_t kc = (P * gx * gy + 152 * 4 - 1) / (152 * 4);
      kc = (kc + FBK - 1) / FBK * FBK;
      if (kc < 1024) kc = 1024;
      a.kchunk = kc;
      dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)((P + kc - 1) / kc));
      k_conv_fast<MODE_WGRAD, 2, 4><<<grid, 256, 0, s->stream>>>(a, wt);
    }
    return cudaGetLastError();
  }
  if (mode == MODE_FWD) {
    dim3 grid((unsigned)((P + BM - 1) / BM), (unsigned)((a.cout + BN - 1) / BN));
    k_conv<MODE_FWD><<<grid, kThreads, 0, s->stream>>>(a);
  } else if (mode == MODE_BWD_DATA) {
    dim3 grid((unsigned)((P + BM - 1) / BM), (unsigned)((a.cin + BN - 1) / BN));
    k_conv<MODE_BWD_DATA><<<grid, kThreads, 0, s->stream>>>(a);
  } else {
    a.kchunk = 4096;
    dim3 grid((unsigned)((a.cout + BM - 1) / BM), (unsigned)((9 * a.cin + BN - 1) / BN),
              (unsigned)((P + a.kchunk - 1) / a.kchunk));
    k_conv<MODE_WGRAD><<<grid, kThreads, 0, s->stream>>>(a);
  }
  return cudaGetLastError();
}

// BF16 copies (and the transposed and padded copies) of the FP32 masters
cudaError_t refresh_bf16(const nlse_sur* s, bool copy) {
  if (copy) k_to_bf16<<<grid1d(s->nparam), 256, 0, s->stream>>>(s->params, s->pbf, s->nparam);
  for (int l = 1; l < s->L - 1; ++l)
    k_transpose_w<<<grid1d((int64_t)s->C * 9 * s->C), 256, 0, s->stream>>>(s->pbf + s->w_off[l],
                                                                          s->pbfT + s->w_off[l], s->C, s->C);
  k_pad_ends<<<grid1d((int64_t)s->C * 9 * s->pc), 256, 0, s->stream>>>(
      s->pbf + s->w_off[0], s->pbf + s->w_off[s->L - 1], s->params + s->b_off[s->L - 1], s->C, s->pc, s->pw0,
      s->pwL, s->pwLT, s->pbL);
  return cudaGetLastError();
}

// training = false (inference): the inner layers keep only silu(z); true: also silu'(z)
cudaError_t forward(const nlse_sur* s, int nb, const float2* psi_in, bool training) {
  const int64_t P = (int64_t)nb * s->H * s->W;
  k_pack_input<<<grid1d(P * s->pc / 8), 256, 0, s->stream>>>(psi_in, P, s->pc, s->hin);
  cudaError_t e = cudaGetLastError();
  const bf16* x = s->hin;
  for (int l = 0; l < s->L && e == cudaSuccess; ++l) {
    const bool last = l == s->L - 1;
    bf16* h = last ? nullptr : s->h[l];
    e = conv(s, MODE_FWD, l, nb, x, nullptr, last ? s->y : nullptr, h, (training && !last) ? s->sd[l] : nullptr,
             nullptr, nullptr);
    x = h;
  }
  return e;
}

// gradients of the mean squared error into s->grad (zeroed first); loss into s->loss
cudaError_t backward(const nlse_sur* s, int nb, const float2* psi_in, const float2* target) {
  const int64_t P = (int64_t)nb * s->H * s->W;
  cudaError_t e = cudaMemsetAsync(s->grad, 0, sizeof(float) * s->nparam, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->loss, 0, sizeof(double), s->stream);
  if (e != cudaSuccess) return e;
  bf16* dz = s->dzA;   // gradient w.r.t. the current layer's pre-activation
  const int64_t HW = (int64_t)s->H * s->W;
  if (s->mass_weight > 0.0) {
    k_state_mass_res<<<dim3(kMassBlocks, (unsigned)nb), 256, 0, s->stream>>>(psi_in, s->y, s->pc, target, HW,
                                                                             s->mass_part);
    k_mass_coef<<<(nb + 31) / 32, 32, 0, s->stream>>>(s->mass_part, nb, s->mass_weight, s->mstat, s->loss);
  }
  k_mse<<<grid1d(P * s->pc / 8), 256, 0, s->stream>>>(psi_in, s->y, target, P, s->pc, dz, s->loss,
                                                      s->mass_weight > 0.0 ? s->mstat : nullptr, HW);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int l = s->L - 1; l >= 0 && e == cudaSuccess; --l) {
    const bool first = l == 0, last = l == s->L - 1;
    const LayerOps o = layer_ops(s, l);
    const bf16* xin = first ? s->hin : s->h[l - 1];
    if (first || last)
      e = cudaMemsetAsync(s->wscr, 0, sizeof(float) * ((size_t)9 * s->pc * s->C + s->pc), s->stream);
    bool bias_done = false;
    if (e == cudaSuccess) e = conv(s, MODE_WGRAD, l, nb, xin, dz, nullptr, nullptr, nullptr, nullptr, nullptr, &bias_done);
    if (e != cudaSuccess) break;
    if (!bias_done) k_bias_grad<<<4 * s->num_sms, 256, 0, s->stream>>>(dz, P, o.cout, o.cout, o.db);
    if (first || last)
      k_unpad_grad<<<grid1d((int64_t)9 * kIn * s->C + s->C), 256, 0, s->stream>>>(
          s->wscr, s->grad + s->w_off[l], s->grad + s->b_off[l], s->C, s->pc, first ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if (l > 0) {
      bf16* dzp = (dz == s->dzA) ? s->dzB : s->dzA;
      e = conv(s, MODE_BWD_DATA, l, nb, nullptr, dz, nullptr, nullptr, nullptr, s->sd[l - 1], dzp);
      dz = dzp;
    }
  }
  return e;
}

// Read and clear the device timeout flag (the stream must be idle).
bool take_err(const nlse_sur* s) {
  int v = 0;
  if (cudaMemcpy(&v, s->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
  if (v) cudaMemset(s->err, 0, sizeof(int));
  return v != 0;
}

}  // namespace

extern "C" {

int nlse_sur_set_kernel(nlse_sur_t s, int tensor_core_gen) {
  if (!s) return sfail(NLSE_EINVAL, "NULL surrogate");
  if (tensor_core_gen != 0 && tensor_core_gen != 1) return sfail(NLSE_EINVAL, "kernel choice must be 0 or 1");
  s->use_tc = tensor_core_gen;
  return NLSE_OK;
}

int nlse_sur_sync(nlse_sur_t s) {
  if (!s) return sfail(NLSE_EINVAL, "NULL surrogate");
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return sfail(NLSE_ECUDA, cudaGetErrorString(e));
  if (take_err(s)) return sfail(NLSE_ETIMEOUT, "a tensor-core convolution wait ran out");
  return NLSE_OK;
}

size_t nlse_sur_param_count(int channels, int layers) {
  if (channels < 1 || channels > 256 || layers < 2 || layers > kMaxLayers) return 0;
  return (size_t)param_count(channels, layers);
}

size_t nlse_sur_workspace_bytes(int H, int W, int channels, int layers, int max_batch) {
  if (H < 1 || W < 1 || max_batch < 1 || nlse_sur_param_count(channels, layers) == 0) return 0;
  return ws_bytes(H, W, channels, layers, max_batch);
}

int nlse_sur_create(nlse_sur_t* out, int H, int W, int channels, int layers, const int* dilations, int max_batch,
                    float* params, void* workspace, size_t ws, void* stream) {
  if (!out) return sfail(NLSE_EINVAL, "out is NULL");
  *out = nullptr;
  const size_t need = nlse_sur_workspace_bytes(H, W, channels, layers, max_batch);
  if (need == 0 || !dilations || !params) return sfail(NLSE_EINVAL, "bad surrogate shape or NULL pointer");
  if (!workspace || (uintptr_t)workspace % 256) return sfail(NLSE_EINVAL, "workspace must be 256-byte aligned");
  if (ws < need) return sfail(NLSE_ENOMEM, "surrogate workspace too small");
  for (int l = 0; l < layers; ++l)
    if (dilations[l] < 1 || dilations[l] > 64) return sfail(NLSE_EINVAL, "dilations must be 1..64");
  nlse_sur* s = new nlse_sur();
  s->H = H; s->W = W; s->C = channels; s->L = layers; s->max_batch = max_batch;
  for (int l = 0; l < layers; ++l) s->dil[l] = dilations[l];
  s->params = params;
  s->nparam = param_count(channels, layers);
  s->stream = (cudaStream_t)stream;
  int64_t off = 0;
  for (int l = 0; l < layers; ++l) {
    const int ci = cin_of(s, l), co = cout_of(s, l);
    s->w_off.push_back(off);
    off += (int64_t)co * 9 * ci;
    s->b_off.push_back(off);
    off += co;
  }
  const int64_t P = (int64_t)max_batch * H * W;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  char* base = (char*)workspace;
  size_t o = 0;
  s->pbf = (bf16*)(base + o); o = al(o + s->nparam * 2);
  s->pbfT = (bf16*)(base + o); o = al(o + s->nparam * 2);
  s->grad = (float*)(base + o); o = al(o + s->nparam * 4);
  s->m1 = (float*)(base + o); o = al(o + s->nparam * 4);
  s->m2 = (float*)(base + o); o = al(o + s->nparam * 4);
  s->loss = (double*)(base + o); o = al(o + 64);
  s->mass_part = (double*)(base + o); o = al(o + (size_t)max_batch * kMassBlocks * 2 * 8);
  s->mstat = (double*)(base + o); o = al(o + (size_t)max_batch * 2 * 8);
  s->mass_weight = 0.0;
  s->amax_part = (float*)(base + o); o = al(o + (size_t)max_batch * kMassBlocks * 4);
  s->xnoisy = (float2*)(base + o); o = al(o + P * 8);
  s->err = (int*)(base + o); o = al(o + 16);
  s->pc = pad_width(channels);
  const int pc = s->pc;
  s->hin = (bf16*)(base + o); o = al(o + P * pc * 2);
  s->pw0 = (bf16*)(base + o); o = al(o + (size_t)channels * 9 * pc * 2);
  s->pwL = (bf16*)(base + o); o = al(o + (size_t)channels * 9 * pc * 2);
  s->pwLT = (bf16*)(base + o); o = al(o + (size_t)channels * 9 * pc * 2);
  s->pbL = (float*)(base + o); o = al(o + pc * 4);
  s->wscr = (float*)(base + o); o = al(o + ((size_t)channels * 9 * pc + pc) * 4);
  s->wgpart = (float*)(base + o); o = al(o + (channels == 64 ? (size_t)kWgMaxParts * kWgPart * 4 : 0));
  s->y = (float*)(base + o); o = al(o + P * pc * 4);
  for (int l = 0; l < layers - 1; ++l) { s->sd.push_back((bf16*)(base + o)); o = al(o + P * channels * 2); }
  for (int l = 0; l < layers - 1; ++l) { s->h.push_back((bf16*)(base + o)); o = al(o + P * channels * 2); }
  const int64_t cz = channels > pc ? channels : pc;
  s->dzA = (bf16*)(base + o); o = al(o + P * cz * 2);
  s->dzB = (bf16*)(base + o); o = al(o + P * cz * 2);
  s->adam_t = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  s->num_sms = 1;
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
  s->use_tc = 1;
  cudaError_t e = cudaSuccess;
  {
    const void* fns[4] = {(const void*)k_conv_tc<MODE_FWD, 0>, (const void*)k_conv_tc<MODE_BWD_DATA, 0>,
                          (const void*)k_conv_tc<MODE_FWD, 1>, (const void*)k_conv_tc<MODE_BWD_DATA, 1>};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
      e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->m1, 0, s->nparam * 4, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->m2, 0, s->nparam * 4, s->stream);
  if (e == cudaSuccess) e = refresh_bf16(s, true);
  if (e != cudaSuccess) {
    delete s;
    return sfail(NLSE_ECUDA, cudaGetErrorString(e));
  }
  *out = s;
  return NLSE_OK;
}

int nlse_sur_init(nlse_sur_t s, uint64_t seed) {
  if (!s) return sfail(NLSE_EINVAL, "NULL surrogate");
  s->seed = seed;
  for (int l = 0; l < s->L; ++l) {
    const int ci = cin_of(s, l), co = cout_of(s, l);
    // uniform He-style scale sqrt(6 / fan_in); the output layer starts small (near-identity residual)
    const float sc = (l == s->L - 1 ? 0.1f : 1.f) * sqrtf(6.f / float(9 * ci));
    const int64_t nw = (int64_t)co * 9 * ci;
    k_init<<<grid1d(nw), 256, 0, s->stream>>>(s->params, s->w_off[l], nw, sc, seed);
    cudaMemsetAsync(s->params + s->b_off[l], 0, sizeof(float) * co, s->stream);
  }
  refresh_bf16(s, true);
  s->adam_t = 0;
  cudaMemsetAsync(s->m1, 0, s->nparam * 4, s->stream);
  cudaMemsetAsync(s->m2, 0, s->nparam * 4, s->stream);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NLSE_OK : sfail(NLSE_ECUDA, cudaGetErrorString(e));
}

int nlse_sur_sync_params(nlse_sur_t s) {
  if (!s) return sfail(NLSE_EINVAL, "NULL surrogate");
  cudaError_t e = refresh_bf16(s, true);
  return e == cudaSuccess ? NLSE_OK : sfail(NLSE_ECUDA, cudaGetErrorString(e));
}

int nlse_sur_forward(nlse_sur_t s, int nb, const void* psi_in, void* psi_out, int project_mass, double* masses_out) {
  if (!s || !psi_in || !psi_out) return sfail(NLSE_EINVAL, "NULL argument");
  if (nb < 1 || nb > s->max_batch) return sfail(NLSE_EINVAL, "batch outside 1..max_batch");
  cudaError_t e = forward(s, nb, (const float2*)psi_in, false);
  if (e == cudaSuccess) {
    const int64_t P = (int64_t)nb * s->H * s->W;
    k_residual<<<grid1d(P), 256, 0, s->stream>>>((const float2*)psi_in, s->y, P, s->pc, (float2*)psi_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && (project_mass || masses_out)) {
    const int64_t HW = (int64_t)s->H * s->W;
    const dim3 grid(kMassBlocks, (unsigned)nb);
    k_state_mass<<<grid, 256, 0, s->stream>>>((const float2*)psi_in, (const float2*)psi_out, HW, s->mass_part);
    if (masses_out) k_state_sums<<<(nb + 31) / 32, 32, 0, s->stream>>>(s->mass_part, nb, masses_out);
    if (project_mass) k_project<<<grid, 256, 0, s->stream>>>((float2*)psi_out, HW, s->mass_part);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? NLSE_OK : sfail(NLSE_ECUDA, cudaGetErrorString(e));
}

int nlse_sur_set_mass_weight(nlse_sur_t s, double mass_weight) {
  if (!s) return sfail(NLSE_EINVAL, "NULL surrogate");
  if (!(mass_weight >= 0.0) || !isfinite(mass_weight)) return sfail(NLSE_EINVAL, "mass weight must be >= 0");
  s->mass_weight = mass_weight;
  return NLSE_OK;
}

int nlse_sur_compare(nlse_sur_t s, int nb, const void* a, const void* b, double* rel_l2_host) {
  if (!s || !a || !b || !rel_l2_host) return sfail(NLSE_EINVAL, "NULL argument");
  if (nb < 1 || nb > s->max_batch) return sfail(NLSE_EINVAL, "batch outside 1..max_batch");
  const int64_t HW = (int64_t)s->H * s->W;
  k_state_diff<<<dim3(kMassBlocks, (unsigned)nb), 256, 0, s->stream>>>((const float2*)a, (const float2*)b, HW,
                                                                       s->mass_part);
  k_state_sums<<<(nb + 31) / 32, 32, 0, s->stream>>>(s->mass_part, nb, s->mstat);
  cudaError_t e = cudaGetLastError();
  std::vector<double> sums(2 * (size_t)nb);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sums.data(), s->mstat, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost,
                                            s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return sfail(NLSE_ECUDA, cudaGetErrorString(e));
  for (int i = 0; i < nb; ++i)
    rel_l2_host[i] = sums[2 * i + 1] > 0.0 ? sqrt(sums[2 * i] / sums[2 * i + 1]) : (sums[2 * i] > 0.0 ? INFINITY : 0.0);
  return NLSE_OK;
}

int nlse_sur_gradients(nlse_sur_t s, int nb, const void* psi_in, const void* psi_target, float* grad_out,
                       double* loss_out) {
  if (!s || !psi_in || !psi_target) return sfail(NLSE_EINVAL, "NULL argument");
  if (nb < 1 || nb > s->max_batch) return sfail(NLSE_EINVAL, "batch outside 1..max_batch");
  cudaError_t e = forward(s, nb, (const float2*)psi_in, true);
  if (e == cudaSuccess) e = backward(s, nb, (const float2*)psi_in, (const float2*)psi_target);
  if (e == cudaSuccess && grad_out)
    e = cudaMemcpyAsync(grad_out, s->grad, sizeof(float) * s->nparam, cudaMemcpyDeviceToDevice, s->stream);
  double l = 0.0;
  if (e == cudaSuccess && loss_out) {
    e = cudaMemcpyAsync(&l, s->loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    *loss_out = l;
    if (e == cudaSuccess && take_err(s)) return sfail(NLSE_ETIMEOUT, "a tensor-core convolution wait ran out");
  }
  return e == cudaSuccess ? NLSE_OK : sfail(NLSE_ECUDA, cudaGetErrorString(e));
}

int nlse_sur_train_step(nlse_sur_t s, int nb, const void* psi_in, const void* psi_target, float lr, float noise,
                        double* loss_out) {
  if (!s || !psi_in || !psi_target) return sfail(NLSE_EINVAL, "NULL argument");
  if (nb < 1 || nb > s->max_batch) return sfail(NLSE_EINVAL, "batch outside 1..max_batch");
  if (!(noise >= 0.f) || !(lr > 0.f)) return sfail(NLSE_EINVAL, "lr must be > 0 and noise >= 0");
  const void* x = psi_in;
  if (noise > 0.f) {
    const int64_t HW = (int64_t)s->H * s->W;
    const dim3 grid(kMassBlocks, (unsigned)nb);
    k_state_amax<<<grid, 256, 0, s->stream>>>((const float2*)psi_in, HW, s->amax_part);
    k_add_noise<<<grid, 256, 0, s->stream>>>((const float2*)psi_in, HW, nb, s->amax_part, noise,
                                             splitmix64(s->seed ^ (0x5851F42D4C957F2Dull * (uint64_t)(s->adam_t + 1))),
                                             s->xnoisy);
    const cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return sfail(NLSE_ECUDA, cudaGetErrorString(e0));
    x = s->xnoisy;
  }
  int rc = nlse_sur_gradients(s, nb, x, psi_target, nullptr, nullptr);
  if (rc != NLSE_OK) return rc;
  s->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, float(s->adam_t)), c2 = 1.f - powf(b2, float(s->adam_t));
  k_adam<<<grid1d(s->nparam), 256, 0, s->stream>>>(s->params, s->grad, s->m1, s->m2, s->pbf, s->nparam, lr, b1, b2,
                                                   1e-8f, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = refresh_bf16(s, false);
  if (e == cudaSuccess && loss_out) {
    double l = 0.0;
    e = cudaMemcpyAsync(&l, s->loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    *loss_out = l;
    if (e == cudaSuccess && take_err(s)) return sfail(NLSE_ETIMEOUT, "a tensor-core convolution wait ran out");
  }
  return e == cudaSuccess ? NLSE_OK : sfail(NLSE_ECUDA, cudaGetErrorString(e));
}

int nlse_sur_destroy(nlse_sur_t s) {
  delete s;
  return NLSE_OK;
}

}  // extern "C"
