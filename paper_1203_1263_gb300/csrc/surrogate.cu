// Learned surrogate: a residual convolutional network that advances a 2D
// complex state by one window of RK4 steps, trained and run on the GPU by the
// kernels in this file (BF16 tensor-core products with FP32 accumulation).
//
// Network (channels-last activations, H x W grid, batch nb):
//   h_{-1} = (Re psi, Im psi)                                    2 channels
//   z_l = conv3x3_{dil_l}(h_{l-1}) + b_l,  h_l = silu(z_l)       l = 0 .. L-2, C channels
//   y   = conv3x3_{dil_{L-1}}(h_{L-2}) + b_{L-1}                 2 channels
//   psi_out = psi_in + (y_0 + i y_1)
// with zero padding at the grid edges.  Parameters are FP32 masters; the
// products use BF16 copies.  Every convolution (forward, backward-data,
// weight-gradient) is one implicit GEMM, C[M x N] += A[M x K] B[K x N], whose
// A and B tiles are gathered from the activations and weights into shared
// memory as BF16 and multiplied with mma.sync.m16n8k16 (FP32 accumulators):
//   forward        M = pixels, N = Cout, K = 9 Cin: A[p,(t,ci)] = h[p + d o_t, ci], B[(t,ci),co] = W[co,t,ci]
//   backward-data  M = pixels, N = Cin,  K = 9 Cout: A[p,(t,co)] = dz[p - d o_t, co], B[(t,co),ci] = W[co,t,ci]
//   weight-grad    M = Cout,   N = 9 Cin, K = pixels: A[co,p] = dz[p, co], B[p,(t,ci)] = h[p + d o_t, ci]
// Loss: mean squared error of psi_out against the target (Re and Im parts);
// optimiser: Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "../../include/nlse.h"

namespace nlse {
void record_last_error(const char* msg);
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
  float* z;             // forward: pre-activation out (FP32), or the raw output of the last layer
  bf16* h;              // forward: silu(z) out (BF16); nullptr for the last layer
  const float* zprev;   // backward-data: pre-activation of the previous layer (for silu'), nullptr = none
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
          a.z[m * a.cout + n] = zv;
          if (a.h) a.h[m * a.cout + n] = __float2bfloat16_rn(silu(zv));
        } else if (MODE == MODE_BWD_DATA) {
          const float d = a.zprev ? v * dsilu(a.zprev[m * a.cin + n]) : v;
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
            *reinterpret_cast<float2*>(&a.z[m * a.cout + n]) = make_float2(z0, z1);
            if (a.h)
              *reinterpret_cast<__nv_bfloat162*>(&a.h[m * a.cout + n]) = __floats2bfloat162_rn(silu(z0), silu(z1));
          } else if (n < N) {
            const float z0 = v0 + a.bias[n];
            a.z[m * a.cout + n] = z0;
            if (a.h) a.h[m * a.cout + n] = __float2bfloat16_rn(silu(z0));
          }
        } else if (MODE == MODE_BWD_DATA) {
          if (n + 1 < N) {
            float d0 = v0, d1 = v1;
            if (a.zprev) {
              const float2 zp = *reinterpret_cast<const float2*>(&a.zprev[m * a.cin + n]);
              d0 *= dsilu(zp.x);
              d1 *= dsilu(zp.y);
            }
            *reinterpret_cast<__nv_bfloat162*>(&a.dzprev[m * a.cin + n]) = __floats2bfloat162_rn(d0, d1);
          } else if (n < N) {
            const float d0 = a.zprev ? v0 * dsilu(a.zprev[m * a.cin + n]) : v0;
            a.dzprev[m * a.cin + n] = __float2bfloat16_rn(d0);
          }
        } else {
          if (n < N) atomicAdd(&a.dw[m * N + n], v0);
          if (n + 1 < N) atomicAdd(&a.dw[m * N + n + 1], v1);
        }
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

// complex state -> 2-channel BF16 input; also FP32 copy of the state for the residual
__global__ void k_pack_input(const float2* __restrict__ psi, int64_t P, bf16* __restrict__ h) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = psi[p];
    h[2 * p] = __float2bfloat16_rn(v.x);
    h[2 * p + 1] = __float2bfloat16_rn(v.y);
  }
}

// psi_out = psi_in + y
__global__ void k_residual(const float2* __restrict__ psi, const float* __restrict__ y, int64_t P,
                           float2* __restrict__ out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = psi[p];
    out[p] = make_float2(v.x + y[2 * p], v.y + y[2 * p + 1]);
  }
}

// MSE loss (FP64 partial sums) and its gradient w.r.t. y, written as BF16 dz of the last layer
__global__ void k_mse(const float2* __restrict__ psi, const float* __restrict__ y, const float2* __restrict__ target,
                      int64_t P, bf16* __restrict__ dz, double* __restrict__ loss_acc) {
  __shared__ double red[256];
  double s = 0.0;
  const float scale = 2.f / float(2 * P);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = psi[p], t = target[p];
    const float ex = v.x + y[2 * p] - t.x, ey = v.y + y[2 * p + 1] - t.y;
    s += double(ex) * ex + double(ey) * ey;
    dz[2 * p] = __float2bfloat16_rn(scale * ex);
    dz[2 * p + 1] = __float2bfloat16_rn(scale * ey);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss_acc, red[0] / double(2 * P));
}

// db[c] = sum over pixels of dz[p, c]  (one block per channel)
__global__ void k_bias_grad(const bf16* __restrict__ dz, int64_t P, int C, float* __restrict__ db) {
  __shared__ float red[256];
  float s = 0.f;
  for (int64_t p = threadIdx.x; p < P; p += blockDim.x) s += __bfloat162float(dz[p * C + blockIdx.x]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[blockIdx.x] += red[0];
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
  bf16* hin;                      // input activation, 2 channels
  std::vector<float*> z;          // pre-activations, layer 0..L-1 (last: y, 2 channels)
  std::vector<bf16*> h;           // activations, layer 0..L-2
  bf16* dzA;                      // gradient ping-pong buffers (C channels)
  bf16* dzB;
  int64_t adam_t;
};

namespace {

int cin_of(const nlse_sur* s, int l) { return l == 0 ? 2 : s->C; }
int cout_of(const nlse_sur* s, int l) { return l == s->L - 1 ? 2 : s->C; }

int64_t param_count(int C, int L) {
  int64_t n = 0;
  for (int l = 0; l < L; ++l) {
    const int ci = l == 0 ? 2 : C, co = l == L - 1 ? 2 : C;
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
  off = al(off + P * 2 * 2);         // hin
  for (int l = 0; l < L; ++l) off = al(off + P * (l == L - 1 ? 2 : C) * 4);   // z
  for (int l = 0; l < L - 1; ++l) off = al(off + P * C * 2);                   // h
  off = al(off + P * C * 2);         // dzA
  off = al(off + P * C * 2);         // dzB
  return off;
}

bool fast_ok(int mode, int cin, int cout) {
  if (mode == MODE_FWD) return cin % 8 == 0 && cout % 2 == 0;
  if (mode == MODE_BWD_DATA) return cout % 8 == 0 && cin % 2 == 0;
  return cout % 8 == 0 && cin % 8 == 0;
}

cudaError_t conv(const nlse_sur* s, int mode, int l, int nb, const bf16* x, const bf16* dz, float* z, bf16* h,
                 const float* zprev, bf16* dzprev, float* dw) {
  ConvArgs a;
  memset(&a, 0, sizeof(a));
  a.g = {nb, s->H, s->W};
  a.cin = cin_of(s, l);
  a.cout = cout_of(s, l);
  a.dil = s->dil[l];
  a.x = x;
  a.dz = dz;
  a.w = s->pbf + s->w_off[l];
  a.bias = s->params + s->b_off[l];
  a.z = z;
  a.h = h;
  a.zprev = zprev;
  a.dzprev = dzprev;
  a.dw = dw;
  const int64_t P = (int64_t)nb * s->H * s->W;
  const bf16* wt = s->pbfT + s->w_off[l];
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

// BF16 copies (and the transposed copies) of the FP32 masters
cudaError_t refresh_bf16(const nlse_sur* s, bool copy) {
  if (copy) k_to_bf16<<<grid1d(s->nparam), 256, 0, s->stream>>>(s->params, s->pbf, s->nparam);
  for (int l = 0; l < s->L; ++l) {
    const int ci = cin_of(s, l), co = cout_of(s, l);
    k_transpose_w<<<grid1d((int64_t)co * 9 * ci), 256, 0, s->stream>>>(s->pbf + s->w_off[l], s->pbfT + s->w_off[l],
                                                                     ci, co);
  }
  return cudaGetLastError();
}

cudaError_t forward(const nlse_sur* s, int nb, const float2* psi_in) {
  const int64_t P = (int64_t)nb * s->H * s->W;
  k_pack_input<<<grid1d(P), 256, 0, s->stream>>>(psi_in, P, s->hin);
  cudaError_t e = cudaGetLastError();
  const bf16* x = s->hin;
  for (int l = 0; l < s->L && e == cudaSuccess; ++l) {
    bf16* h = (l < s->L - 1) ? s->h[l] : nullptr;
    e = conv(s, MODE_FWD, l, nb, x, nullptr, s->z[l], h, nullptr, nullptr, nullptr);
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
  k_mse<<<grid1d(P), 256, 0, s->stream>>>(psi_in, s->z[s->L - 1], target, P, dz, s->loss);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int l = s->L - 1; l >= 0 && e == cudaSuccess; --l) {
    const bf16* xin = (l == 0) ? s->hin : s->h[l - 1];
    e = conv(s, MODE_WGRAD, l, nb, xin, dz, nullptr, nullptr, nullptr, nullptr, s->grad + s->w_off[l]);
    if (e != cudaSuccess) break;
    k_bias_grad<<<cout_of(s, l), 256, 0, s->stream>>>(dz, P, cout_of(s, l), s->grad + s->b_off[l]);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if (l > 0) {
      bf16* dzp = (dz == s->dzA) ? s->dzB : s->dzA;
      e = conv(s, MODE_BWD_DATA, l, nb, nullptr, dz, nullptr, nullptr, s->z[l - 1], dzp, nullptr);
      dz = dzp;
    }
  }
  return e;
}

}  // namespace

extern "C" {

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
  s->hin = (bf16*)(base + o); o = al(o + P * 2 * 2);
  for (int l = 0; l < layers; ++l) { s->z.push_back((float*)(base + o)); o = al(o + P * cout_of(s, l) * 4); }
  for (int l = 0; l < layers - 1; ++l) { s->h.push_back((bf16*)(base + o)); o = al(o + P * channels * 2); }
  s->dzA = (bf16*)(base + o); o = al(o + P * channels * 2);
  s->dzB = (bf16*)(base + o); o = al(o + P * channels * 2);
  s->adam_t = 0;
  cudaError_t e = cudaMemsetAsync(s->m1, 0, s->nparam * 4, s->stream);
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

int nlse_sur_forward(nlse_sur_t s, int nb, const void* psi_in, void* psi_out, int project_mass) {
  if (!s || !psi_in || !psi_out) return sfail(NLSE_EINVAL, "NULL argument");
  if (nb < 1 || nb > s->max_batch) return sfail(NLSE_EINVAL, "batch outside 1..max_batch");
  cudaError_t e = forward(s, nb, (const float2*)psi_in);
  if (e == cudaSuccess) {
    const int64_t P = (int64_t)nb * s->H * s->W;
    k_residual<<<grid1d(P), 256, 0, s->stream>>>((const float2*)psi_in, s->z[s->L - 1], P, (float2*)psi_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && project_mass) {
    const int64_t HW = (int64_t)s->H * s->W;
    const dim3 grid(kMassBlocks, (unsigned)nb);
    k_state_mass<<<grid, 256, 0, s->stream>>>((const float2*)psi_in, (const float2*)psi_out, HW, s->mass_part);
    k_project<<<grid, 256, 0, s->stream>>>((float2*)psi_out, HW, s->mass_part);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? NLSE_OK : sfail(NLSE_ECUDA, cudaGetErrorString(e));
}

int nlse_sur_gradients(nlse_sur_t s, int nb, const void* psi_in, const void* psi_target, float* grad_out,
                       double* loss_out) {
  if (!s || !psi_in || !psi_target) return sfail(NLSE_EINVAL, "NULL argument");
  if (nb < 1 || nb > s->max_batch) return sfail(NLSE_EINVAL, "batch outside 1..max_batch");
  cudaError_t e = forward(s, nb, (const float2*)psi_in);
  if (e == cudaSuccess) e = backward(s, nb, (const float2*)psi_in, (const float2*)psi_target);
  if (e == cudaSuccess && grad_out)
    e = cudaMemcpyAsync(grad_out, s->grad, sizeof(float) * s->nparam, cudaMemcpyDeviceToDevice, s->stream);
  double l = 0.0;
  if (e == cudaSuccess && loss_out) {
    e = cudaMemcpyAsync(&l, s->loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    *loss_out = l;
  }
  return e == cudaSuccess ? NLSE_OK : sfail(NLSE_ECUDA, cudaGetErrorString(e));
}

int nlse_sur_train_step(nlse_sur_t s, int nb, const void* psi_in, const void* psi_target, float lr, double* loss_out) {
  int rc = nlse_sur_gradients(s, nb, psi_in, psi_target, nullptr, nullptr);
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
  }
  return e == cudaSuccess ? NLSE_OK : sfail(NLSE_ECUDA, cudaGetErrorString(e));
}

int nlse_sur_destroy(nlse_sur_t s) {
  delete s;
  return NLSE_OK;
}

}  // extern "C"
