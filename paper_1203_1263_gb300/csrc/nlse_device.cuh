// Device-side building blocks of the RK4 NLSE stage kernels (sm_103a).
//
// What one stage computes at an interior site c (every index in [1, N-2]):
//   F_c = i [ a Lap Psi_c + (s|Psi_c|^2 - V_c) Psi_c ]                 (Sec. 3.1)
// and then the fused RK4 update of Eq. RK4_GPU for that stage.  Boundary
// sites are updated by the interior site that is their "b-1" neighbour (one
// step inward along every axis on which the boundary site sits on a face),
// with F_b = 0 (Dirichlet, Eq. BCDdt) or F_b = i Im(F_c / Psi_c) Psi_b (MSD,
// Eq. msd).  Every boundary site has exactly one such interior site, so each
// site of the grid is written by exactly one thread per stage.
//
// Laplacian.  Order 2 is the central difference (step 1 of Eqs. 2shoc1d,
// 2d2shocs1, 3d2shocs).  Order 4 is 2SHOC (Eqs. 2shoc1d2, 2d2shocs2,
// 3d2shocs2).  Where every face neighbour of c is interior, 2SHOC equals, in
// exact arithmetic, the axis-separable five-point form
//     Lap_c = sum_axes [16 (Psi_{+1} + Psi_{-1}) - (Psi_{+2} + Psi_{-2}) - 30 Psi_c] / (12 h^2)
// (expand D = Lap_CD Psi in the step-2 stencil: the cross terms of the
// neighbour D's cancel against the edge-diagonal Psi terms), which needs no
// D array and a third of the arithmetic.  Where a face neighbour b of c is a
// boundary site, 2SHOC uses the boundary Laplacian form D_b (Eq. BCDlap or
// Eq. BCMSDlap) instead of the central difference at b; the same five-point
// form still holds if the missing value Psi_{+-2} beyond the wall is replaced
// by the "ghost" g that makes the central difference at b equal D_b:
//     g = h^2 D_b - Psi_c - sum_{in-face neighbours of b} Psi + 2d Psi_b.
// So one code path covers interior and wall-adjacent sites.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace nlse {

enum { BC_DIRICHLET = 0, BC_MSD = 1 };

template <class R> struct V2;
template <> struct V2<double> { using t = double2; };
template <> struct V2<float> { using t = float2; };

// Precision traits: R = arithmetic type, C = stored complex type of the stage
// arrays, VR = stored type of V, M = stored type of the master Psi^n.
struct P64 { using R = double; using C = double2; using VR = double; using M = double2; };
struct P32 { using R = float;  using C = float2;  using VR = float;  using M = float2;  };
struct PMix { using R = float; using C = float2;  using VR = float;  using M = double2; };
// FP64 evaluation over FP32 / mixed storage (energy of the FP32 forms)
struct E32 { using R = double; using C = float2;  using VR = float;  using M = float2;  };
struct EMix { using R = double; using C = double2; using VR = float; using M = double2; };

template <class R, class C>
__device__ __forceinline__ typename V2<R>::t ld2(const C* __restrict__ p, int64_t i) {
  const C v = __ldg(p + i);
  return {R(v.x), R(v.y)};
}
template <class R, class VR>
__device__ __forceinline__ R ldv(const VR* __restrict__ V, int64_t i) {
  return V ? R(__ldg(V + i)) : R(0);
}

// The grid, the physics and the field a Laplacian is taken of.
template <class T>
struct Field {
  using R = typename T::R;
  int n[3];          // extents, axis D-1 fastest
  int m[3];          // interior extents n - 2
  int64_t st[3];     // strides in sites
  int64_t ninterior;
  R a, s;
  R h2_over_a;       // h^2 / a
  R cL;              // a / (12 h^2) for order 4, a / h^2 for order 2
  R tiny;            // MSD guard on |Psi_{b-1}|^2
  int bc;
  const typename T::VR* V;
  const typename T::C* in;   // the field (stage input Psi)
};

// Operand access for the stencil.  An accessor is positioned at one interior
// site c and returns Psi at c plus small offsets: at1(k, s) = Psi(c + s e_k),
// at2(k, s, j, t) = Psi(c + s e_k + t e_j), atv(o) = Psi(c + sum_k o_k e_k).
// GAcc reads global memory; the tiled kernels supply shared-memory accessors.
// The arithmetic below never depends on which accessor is used.
template <class T, int D>
struct GAcc {
  using R = typename T::R;
  using C2 = typename V2<R>::t;
  const Field<T>& f;
  int64_t c;
  __device__ __forceinline__ GAcc(const Field<T>& f_, int64_t c_) : f(f_), c(c_) {}
  __device__ __forceinline__ C2 at0() const { return ld2<R>(f.in, c); }
  __device__ __forceinline__ C2 at1(int k, int s) const { return ld2<R>(f.in, c + s * f.st[k]); }
  __device__ __forceinline__ C2 at2(int k, int s, int j, int t) const {
    return ld2<R>(f.in, c + s * f.st[k] + t * f.st[j]);
  }
  __device__ __forceinline__ C2 atv(const int* o) const {
    int64_t q = c;
#pragma unroll
    for (int k = 0; k < D; ++k) q += o[k] * f.st[k];
    return ld2<R>(f.in, q);
  }
};

// h^2 D_b at the face boundary site nb = c + dir e_k (Eqs. BCDlap, BCMSDlap),
// then the ghost value beyond the wall.
template <class T, int D, class Acc>
__device__ __forceinline__ typename V2<typename T::R>::t ghost(const Field<T>& f, const Acc& acc, int k, int dir,
                                                               int64_t c, typename V2<typename T::R>::t pc,
                                                               typename V2<typename T::R>::t dh_c,
                                                               typename T::R Nc) {
  using R = typename T::R;
  using C2 = typename V2<R>::t;
  const C2 pb = acc.at1(k, dir);
  const R Nb = f.s * (pb.x * pb.x + pb.y * pb.y) - ldv<R>(f.V, c + dir * f.st[k]);
  R fac;
  if (f.bc == BC_DIRICHLET) {
    fac = -f.h2_over_a * Nb;
  } else {
    const R m2 = pc.x * pc.x + pc.y * pc.y;
    const R ratio = (m2 > f.tiny) ? (dh_c.x * pc.x + dh_c.y * pc.y) / m2 : R(0);
    fac = ratio + f.h2_over_a * (Nc - Nb);
  }
  C2 g = {fac * pb.x - pc.x + R(2 * D) * pb.x, fac * pb.y - pc.y + R(2 * D) * pb.y};
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (j == k) continue;
    const C2 u = acc.at2(k, dir, j, 1);
    const C2 w = acc.at2(k, dir, j, -1);
    g.x -= u.x + w.x;
    g.y -= u.y + w.y;
  }
  return g;
}

// a * Lap(Psi) at interior site c with multi-index idx.
template <class T, int D, int ORDER, class Acc>
__device__ __forceinline__ typename V2<typename T::R>::t a_lap(const Field<T>& f, const Acc& acc, const int* idx,
                                                               int64_t c, typename V2<typename T::R>::t pc,
                                                               typename T::R Nc) {
  using R = typename T::R;
  using C2 = typename V2<R>::t;
  C2 s1 = {R(0), R(0)};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const C2 u = acc.at1(k, 1);
    const C2 w = acc.at1(k, -1);
    s1.x += u.x + w.x;
    s1.y += u.y + w.y;
  }
  if constexpr (ORDER == 2) {
    return {f.cL * (s1.x - R(2 * D) * pc.x), f.cL * (s1.y - R(2 * D) * pc.y)};
  }
  const C2 dh = {s1.x - R(2 * D) * pc.x, s1.y - R(2 * D) * pc.y};   // h^2 D_c
  C2 s2 = {R(0), R(0)};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const C2 lo = (idx[k] >= 2) ? acc.at1(k, -2) : ghost<T, D>(f, acc, k, -1, c, pc, dh, Nc);
    const C2 hi = (idx[k] <= f.n[k] - 3) ? acc.at1(k, 2) : ghost<T, D>(f, acc, k, 1, c, pc, dh, Nc);
    s2.x += lo.x + hi.x;
    s2.y += lo.y + hi.y;
  }
  return {f.cL * (R(16) * s1.x - s2.x - R(30 * D) * pc.x), f.cL * (R(16) * s1.y - s2.y - R(30 * D) * pc.y)};
}

// Everything a stage writes, on top of the field it reads.
template <class T>
struct StageArgs {
  Field<T> f;
  const typename T::C* psin;   // Psi^n in stage precision (stage 1: == f.in)
  typename T::C* ktot;         // K_tot
  typename T::C* out;          // Psi_tmp / Psi_out (stages 1-3); F (stage 0)
  typename T::M* master;       // Psi^n master, updated in stage 4
  typename T::C* n32;          // PMix: FP32 copy of Psi^{n+1} written in stage 4
  typename T::R dtc;           // dt/2, dt/2, dt, dt/6 for stages 1..4
  double dt6;                  // dt/6 in FP64 (PMix stage 4)
  int stage;                   // 0 = write F only, 1..4 = RK4 stage
  unsigned int* flag;          // bit 0: non-finite Psi
};

template <class T>
__device__ __forceinline__ void rk_update(const StageArgs<T>& A, int64_t i, typename V2<typename T::R>::t F) {
  using R = typename T::R;
  using C = typename T::C;
  switch (A.stage) {
    case 0:
      A.out[i] = C{F.x, F.y};
      break;
    case 1: {  // K_tot = k; Psi_tmp = Psi^n + (dt/2) k
      A.ktot[i] = C{F.x, F.y};
      const C p = A.psin[i];
      A.out[i] = C{fma(A.dtc, F.x, p.x), fma(A.dtc, F.y, p.y)};
      break;
    }
    case 2:
    case 3: {  // K_tot += 2k; Psi_out = Psi^n + (dt/2) k  |  Psi_tmp = Psi^n + dt k
      const C K = A.ktot[i];
      A.ktot[i] = C{fma(R(2), F.x, K.x), fma(R(2), F.y, K.y)};
      const C p = A.psin[i];
      A.out[i] = C{fma(A.dtc, F.x, p.x), fma(A.dtc, F.y, p.y)};
      break;
    }
    default: {  // Psi^{n+1} = Psi^n + (dt/6)(K_tot + k)
      const C K = A.ktot[i];
      const typename T::M p = A.master[i];
      typename T::M q;
      if constexpr (std::is_same<typename T::M, C>::value) {
        q.x = fma(A.dtc, K.x + F.x, p.x);
        q.y = fma(A.dtc, K.y + F.y, p.y);
      } else {  // FP64 accumulator over FP32 stages
        q.x = fma(A.dt6, double(K.x) + double(F.x), double(p.x));
        q.y = fma(A.dt6, double(K.y) + double(F.y), double(p.y));
        A.n32[i] = C{R(q.x), R(q.y)};
      }
      A.master[i] = q;
      if (!(isfinite(q.x) && isfinite(q.y))) atomicOr(A.flag, 1u);
      break;
    }
  }
}

// The full per-site work: F at interior site c, its update, and the update of
// every boundary site whose b-1 neighbour is c.
template <class T, int D, int ORDER, class Acc>
__device__ __forceinline__ void process_site(const StageArgs<T>& A, const Acc& acc, const int* idx, int64_t c) {
  using R = typename T::R;
  using C2 = typename V2<R>::t;
  const Field<T>& f = A.f;
  const C2 pc = acc.at0();
  const R Nc = f.s * (pc.x * pc.x + pc.y * pc.y) - ldv<R>(f.V, c);
  const C2 aL = a_lap<T, D, ORDER>(f, acc, idx, c, pc, Nc);
  const C2 F = {-(aL.y + Nc * pc.y), aL.x + Nc * pc.x};
  rk_update<T>(A, c, F);

  bool near = false;
#pragma unroll
  for (int k = 0; k < D; ++k) near |= (idx[k] == 1) | (idx[k] == f.n[k] - 2);
  if (!near) return;
  R theta = R(0);
  if (f.bc == BC_MSD) {
    const R m2 = pc.x * pc.x + pc.y * pc.y;
    if (m2 > f.tiny) theta = (F.y * pc.x - F.x * pc.y) / m2;
  }
  // boundary sites c + sum_k o_k e_k with o_k in {0} u {-1 if idx==1} u {+1 if idx==n-2}, not all 0
  int opts[D][3], nopt[D];
  int combos = 1;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    nopt[k] = 0;
    opts[k][nopt[k]++] = 0;
    if (idx[k] == 1) opts[k][nopt[k]++] = -1;
    if (idx[k] == f.n[k] - 2) opts[k][nopt[k]++] = 1;
    combos *= nopt[k];
  }
  for (int q = 1; q < combos; ++q) {
    int r = q;
    int o[D];
    int64_t b = c;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
      o[k] = opts[k][r % nopt[k]];
      b += o[k] * f.st[k];
      r /= nopt[k];
    }
    C2 Fb = {R(0), R(0)};
    if (f.bc == BC_MSD) {
      const C2 pb = acc.atv(o);
      Fb = {-theta * pb.y, theta * pb.x};
    }
    rk_update<T>(A, b, Fb);
  }
}

// Host-visible launch entry points (defined in stage_*.cu).
template <class T, int D, int ORDER>
cudaError_t launch_stage(const StageArgs<T>& A, int variant, int tile_cfg, cudaStream_t stream);

}  // namespace nlse
