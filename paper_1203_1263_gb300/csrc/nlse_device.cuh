// Device-side building blocks of the RK4 NLSE stage kernels (sm_103a).
//
// What one stage computes at an interior site c (every index in [1, N-2]):
//   F_c = i [ a Lap Psi_c + (s|Psi_c|^2 - V_c) Psi_c ]                 (Sec. 3.1)
// and then the fused RK4 update of Eq. RK4_GPU for that stage.  Boundary
// sites are updated by the interior site that is their "b-1" neighbour (one
// step inward along every axis on which the boundary site sits on a face),
// with F_b = 0 (Dirichlet, Eq. BCDdt), F_b = i Im(F_c / Psi_c) Psi_b (MSD,
// Eq. msd) or F_b = i (s|Psi_b|^2 - V_b) Psi_b (L0, Eq. BCL0dt).  Every
// boundary site has exactly one such interior site, so each site of the grid
// is written by exactly one thread per stage.
//
// Laplacian.  Order 2 is the central difference (step 1 of Eqs. 2shoc1d,
// 2d2shocs1, 3d2shocs).  Order 4 is 2SHOC (Eqs. 2shoc1d2, 2d2shocs2,
// 3d2shocs2).  Where every face neighbour of c is interior, 2SHOC equals, in
// exact arithmetic, the axis-separable five-point form
//     Lap_c = sum_axes [16 (Psi_{+1} + Psi_{-1}) - (Psi_{+2} + Psi_{-2}) - 30 Psi_c] / (12 h^2)
// (expand D = Lap_CD Psi in the step-2 stencil: the cross terms of the
// neighbour D's cancel against the edge-diagonal Psi terms), which needs no
// D array and a third of the arithmetic.  Where a face neighbour b of c is a
// boundary site, 2SHOC uses the boundary Laplacian form D_b (Eq. BCDlap,
// Eq. BCMSDlap, or D_b = 0 by Eq. BCL0lap) instead of the central difference at b; the same five-point
// form still holds if the missing value Psi_{+-2} beyond the wall is replaced
// by the "ghost" g that makes the central difference at b equal D_b:
//     g = h^2 D_b - Psi_c - sum_{in-face neighbours of b} Psi + 2d Psi_b.
// So one code path covers interior and wall-adjacent sites.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace nlse {

enum { BC_DIRICHLET = 0, BC_MSD = 1, BC_L0 = 2, BC_PERIODIC = 3 };

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

// |z|^2 with one fixed rounding order, so every kernel computes it alike.
template <class C2>
__device__ __forceinline__ auto norm2(const C2 z) -> decltype(z.x) { return fma(z.x, z.x, z.y * z.y); }

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
  int F;             // exact-sum stencil: the reference fraction bits F0 that cLF and V / cLF are scaled by
  const int* Fdev;   // exact-sum stencil: device word holding the fraction bits of the current state
                     //   (derived from max |Psi| every step; nullptr: use F)
  double cLF;        // exact-sum stencil: cL * 2^-F
  R sG;              // exact-sum stencil: s / cLF
  R invcLF;          // exact-sum stencil: 1 / cLF
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
  // fixed-point operands of the exact-sum stencil (FP64 fields only)
  __device__ __forceinline__ longlong2 fx0() const;
  __device__ __forceinline__ longlong2 fx1(int k, int s) const;
  __device__ __forceinline__ longlong2 fx2(int k, int s, int j, int t) const;
  __device__ __forceinline__ int fixF() const { return cur_fix(f); }   // this step's fraction bits
};

// h^2 D_b at the face boundary site nb = c + dir e_k (Eqs. BCDlap, BCMSDlap;
// 0 under L0, Eq. BCL0lap), then the ghost value beyond the wall.
template <class T, int D, class Acc>
__device__ __forceinline__ typename V2<typename T::R>::t ghost(const Field<T>& f, const Acc& acc, int k, int dir,
                                                               int64_t c, typename V2<typename T::R>::t pc,
                                                               typename V2<typename T::R>::t dh_c,
                                                               typename T::R Nc) {
  using R = typename T::R;
  using C2 = typename V2<R>::t;
  const C2 pb = acc.at1(k, dir);
  R fac = R(0);
  if (f.bc != BC_L0) {
    const R Nb = fma(f.s, norm2(pb), -ldv<R>(f.V, c + dir * f.st[k]));
    if (f.bc == BC_DIRICHLET) {
      fac = -f.h2_over_a * Nb;
    } else {
      const R m2 = norm2(pc);
      const R ratio = (m2 > f.tiny) ? fma(dh_c.x, pc.x, dh_c.y * pc.y) / m2 : R(0);
      fac = fma(f.h2_over_a, Nc - Nb, ratio);
    }
  }
  C2 g = {fma(R(2 * D), pb.x, fma(fac, pb.x, -pc.x)), fma(R(2 * D), pb.y, fma(fac, pb.y, -pc.y))};
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

// a * Lap(Psi) at interior site c with multi-index idx; `wall` says whether
// some +-2 neighbour lies beyond a wall (then the ghosts are used).
template <class T, int D, int ORDER, class Acc, bool WALL>
__device__ __forceinline__ typename V2<typename T::R>::t a_lap_body(const Field<T>& f, const Acc& acc, const int* idx,
                                                                    int64_t c, typename V2<typename T::R>::t pc,
                                                                    typename T::R Nc) {
  using R = typename T::R;
  using C2 = typename V2<R>::t;
  // Sums of differences from the centre: Psi_{+-k} - Psi_c is exact for nearby values (Sterbenz), so the
  // large cancellation of the stencil (centre weight 30 d in 2SHOC) happens before any rounding.
  C2 s1 = {R(0), R(0)};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const C2 u = acc.at1(k, 1);
    const C2 w = acc.at1(k, -1);
    s1.x += (u.x - pc.x) + (w.x - pc.x);
    s1.y += (u.y - pc.y) + (w.y - pc.y);
  }
  const C2 dh = s1;   // h^2 D_c
  if constexpr (ORDER == 2) {
    return {f.cL * dh.x, f.cL * dh.y};
  }
  C2 s2 = {R(0), R(0)};
#pragma unroll
  for (int k = 0; k < D; ++k) {
    C2 lo, hi;
    if (!WALL || idx[k] >= 2) lo = acc.at1(k, -2);
    else lo = ghost<T, D>(f, acc, k, -1, c, pc, dh, Nc);
    if (!WALL || idx[k] <= f.n[k] - 3) hi = acc.at1(k, 2);
    else hi = ghost<T, D>(f, acc, k, 1, c, pc, dh, Nc);
    s2.x += (lo.x - pc.x) + (hi.x - pc.x);
    s2.y += (lo.y - pc.y) + (hi.y - pc.y);
  }
  // 16 (s1 + 2d Psi_c) - (s2 + 2d Psi_c) - 30 d Psi_c = 16 s1 - s2
  return {f.cL * fma(R(16), s1.x, -s2.x), f.cL * fma(R(16), s1.y, -s2.y)};
}

template <class T, int D, int ORDER, class Acc>
__device__ __forceinline__ typename V2<typename T::R>::t a_lap_wall(const Field<T>& f, const Acc& acc, const int* idx,
                                                                 int64_t c, typename V2<typename T::R>::t pc,
                                                                 typename T::R Nc) {
  return a_lap_body<T, D, ORDER, Acc, true>(f, acc, idx, c, pc, Nc);
}

template <int D>
__device__ __forceinline__ bool near_wall2(const int* idx, const int* n) {
  bool w = false;
#pragma unroll
  for (int k = 0; k < D; ++k) w |= (idx[k] < 2) | (idx[k] > n[k] - 3);
  return w;
}

template <class T, int D, int ORDER, class Acc>
__device__ __forceinline__ typename V2<typename T::R>::t a_lap(const Field<T>& f, const Acc& acc, const int* idx,
                                                               int64_t c, typename V2<typename T::R>::t pc,
                                                               typename T::R Nc) {
  if (ORDER == 4 && near_wall2<D>(idx, f.n)) return a_lap_wall<T, D, ORDER>(f, acc, idx, c, pc, Nc);
  return a_lap_body<T, D, ORDER, Acc, false>(f, acc, idx, c, pc, Nc);
}

// ---------------------------------------------------------------------------
// Exact-sum stencil for the FP64 path.  GB300 issues FP64 arithmetic at
// 1/75 of the FP32 rate, so the FP64 stage is bound by the FP64 pipe, and
// most of its FP64 instructions are the stencil's additions.  Here every
// stencil operand is converted (on the integer pipe, from its IEEE-754 bits)
// to a 64-bit fixed-point number v * 2^F rounded to nearest; the sums
// 16 s1 - s2 - 30 d Psi_c (or s1 - 2d Psi_c) are then exact integers, and one
// conversion and one multiply by cL 2^-F give a*Lap in FP64.  An operand is
// accepted while |v| 2^F < 2^55; F follows the state so that its largest
// component stays below 2^53 (4x headroom for the stages' intermediate
// states), which keeps all 53 bits of the largest components.  An operand
// outside the range (or Inf/NaN) yields kFixBad and the site falls back to
// the FP64 stencil, so the result is always defined.  Bounds of the sums
// (L = 2^55): a deep site's 16 s1 - s2 - 30 d Psi_c stays below 64 d L
// <= 192 L; a wall ghost is used only while below 2^57 = 4L (else the site
// falls back), so a wall site's sum stays below (32 d + 8 d + 30 d) L <= 210 L;
// both are below 2^63 = 256 L.
// ---------------------------------------------------------------------------
constexpr long long kFixBad = (long long)0x8000000000000000ull;

__device__ __forceinline__ long long fix1(double v, int F) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int e = int((u >> 52) & 0x7FF);
  const long long m = (long long)((u & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull);
  const int sh = e - 1075 + F;
  long long r;
  if (e == 0) return 0;                 // zero or subnormal: below any usable resolution
  if (sh > 2) return kFixBad;           // out of range (|v| 2^F >= 2^55), or Inf / NaN (e = 2047)
  if (sh >= 0) r = m << sh;
  else if (sh >= -54) { const int k = -sh; r = (m + (1ll << (k - 1))) >> k; }
  else r = 0;
  return (u >> 63) ? -r : r;
}
__device__ __forceinline__ longlong2 fix2(double2 v, int F) { return make_longlong2(fix1(v.x, F), fix1(v.y, F)); }

// The fraction bits the exact-sum stencil uses for the current state: F is
// re-derived on the device before every step from the largest component of
// Psi^n (|v| 2^F < 2^53, 4x below the accepted range), so the fixed-point resolution
// 2^-F always follows the state's own scale.  The stencil sums are formed at
// that scale and converted to units of cLF = cL 2^-F0 (F0: the reference
// scale fixed at creation) by an exact power-of-two exponent shift.
template <class T>
__device__ __forceinline__ int cur_fix(const Field<T>& f) { return f.Fdev ? __ldg(f.Fdev) : f.F; }

// Biased IEEE-754 exponent of |v|: 0 for zero and subnormals, 2047 for Inf/NaN.
__device__ __forceinline__ unsigned int expo_bits(double v) { return (unsigned int)(__double2hiint(v) >> 20) & 0x7FFu; }
__device__ __forceinline__ unsigned int expo_bits(float v) { return 0u; }

// Largest biased exponent over a full warp into *p (one atomic per warp, skipped when *p is already as
// large).  Every lane of the warp must call it.
__device__ __forceinline__ void emax_commit(unsigned int* p, unsigned int e) {
  e = __reduce_max_sync(0xffffffffu, e);
  if ((threadIdx.x & 31) == 0 && e > __ldcg(p)) atomicMax(p, e);
}
__device__ __forceinline__ bool fbad(longlong2 v) { return (v.x == kFixBad) | (v.y == kFixBad); }

// The FP64 stencil as an out-of-line call (out-of-range operands).
template <class T, int D, int ORDER, class Acc>
__device__ __forceinline__ double2 a_lap_slow(const Field<T>& f, const Acc& acc, const int* idx, int64_t c, double2 pc,
                                           double Nc) {
  return a_lap_body<T, D, ORDER, Acc, true>(f, acc, idx, c, pc, Nc);
}

// The ghost beyond the wall in fixed point (exact-sum stages): with fac = h^2 D_b / Psi_b (the boundary
// Laplacian form, Eqs. BCDlap, BCMSDlap, BCL0lap) the ghost is g = 2d Psi_b + fac Psi_b - Psi_c -
// sum_{in-face neighbours of b} Psi (see ghost()); only fac and fac Psi_b are formed in FP64, the rest of
// the sum is exact in fixed point.  dh_c = h^2 D_c and m2 = |Psi_c|^2 (0 below the MSD guard)
// come from the caller, once per site.
template <class T, int D, class Acc>
__device__ __forceinline__ longlong2 ghost_fix(const Field<T>& f, const Acc& acc, int k, int dir, int64_t c,
                                               double2 pc, double2 dh_c, double Nc, double m2, int F,
                                               bool* bad) {
  const double2 pb = acc.at1(k, dir);
  double fac = 0.0;
  if (f.bc != BC_L0) {
    const double Nb = fma(f.s, norm2(pb), -ldv<double>(f.V, c + dir * f.st[k]));
    if (f.bc == BC_DIRICHLET) fac = -f.h2_over_a * Nb;
    else fac = fma(f.h2_over_a, Nc - Nb, m2 > 0.0 ? fma(dh_c.x, pc.x, dh_c.y * pc.y) / m2 : 0.0);
  }
  const longlong2 pbf = acc.fx1(k, dir), pcf = acc.fx0(), fp = fix2(make_double2(fac * pb.x, fac * pb.y), F);
  bool b = fbad(pbf) | fbad(pcf) | fbad(fp);
  long long gx = 2 * D * pbf.x + fp.x - pcf.x, gy = 2 * D * pbf.y + fp.y - pcf.y;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (j == k) continue;
    const longlong2 u = acc.fx2(k, dir, j, 1), w = acc.fx2(k, dir, j, -1);
    b |= fbad(u) | fbad(w);
    gx -= u.x + w.x;
    gy -= u.y + w.y;
  }
  // |g| < 4 d 2^55 from its terms; beyond 2^57 the site takes the FP64 stencil (keeps the sum's bound)
  constexpr long long kGhostMax = 1ll << 57;
  b |= (gx >= kGhostMax) | (gx <= -kGhostMax) | (gy >= kGhostMax) | (gy <= -kGhostMax);
  *bad |= b;
  return make_longlong2(gx, gy);
}

// s2 = sum over axes of Psi_{+2} + Psi_{-2} in fixed point at a site next to a
// wall, with the fixed-point ghosts in place of the values beyond the wall.
// dh_c (h^2 D_c) comes from the exact integer sums of the face neighbours.
// Out of line: only wall-adjacent sites call it.
template <class T, int D, class Acc>
__device__ __forceinline__ longlong2 exact_s2_wall(const Field<T>& f, const Acc& acc, const int* idx, int64_t c,
                                                double2 pc, double2 dh, double Nc, double m2, int F,
                                                bool* bad) {
  long long sx = 0, sy = 0;
  bool b = false;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    longlong2 lo, hi;
    if (idx[k] >= 2) lo = acc.fx1(k, -2);
    else lo = ghost_fix<T, D>(f, acc, k, -1, c, pc, dh, Nc, m2, F, &b);
    if (idx[k] <= f.n[k] - 3) hi = acc.fx1(k, 2);
    else hi = ghost_fix<T, D>(f, acc, k, 1, c, pc, dh, Nc, m2, F, &b);
    b |= fbad(lo) | fbad(hi);
    sx += lo.x + hi.x;
    sy += lo.y + hi.y;
  }
  *bad |= b;
  return make_longlong2(sx, sy);
}

// int64 -> double with IEEE-754 round-to-nearest-even, times 2^eadj, on the
// integer pipe (the hardware conversion runs on the FP64 pipe, GB300's
// scarcest unit): the power of two only moves the exponent, so the result is
// the correctly rounded v 2^eadj.  Exact for |v| < 2^53.  A result outside
// the normal range (never for the scales the stencil uses) takes ldexp.
__device__ __forceinline__ double i2d_rn(long long v, int eadj = 0) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ull;
  unsigned long long u = sgn ? 0ull - (unsigned long long)v : (unsigned long long)v;
  int e = 63 - __clzll(u);                 // position of the leading one
  unsigned long long m;
  if (e <= 52) {
    m = u << (52 - e);
  } else {
    const int sh = e - 52;
    m = u >> sh;
    const unsigned long long rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) ++m;
    if (m == (1ull << 53)) { m >>= 1; ++e; }
  }
  const int be = e + 1023 + eadj;
  if (be >= 1 && be <= 2046)
    return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (m & 0x000FFFFFFFFFFFFFull)));
  return ldexp(__longlong_as_double((long long)(sgn | ((unsigned long long)(e + 1023) << 52) |
                                                (m & 0x000FFFFFFFFFFFFFull))), eadj);
}

// The exact-sum Laplacian in units of cLF = cL 2^-F (the exact integer sum
// itself, rounded once to FP64); Ng = N_c / cLF.  Sites with an operand
// outside the fixed-point range take the FP64 stencil, rescaled.
template <class T, int D, int ORDER, class Acc>
__device__ __forceinline__ double2 a_lap_exact(const Field<T>& f, const Acc& acc, const int* idx, int64_t c,
                                               double2 pc, double Ng, double m2) {
  static_assert(std::is_same<typename T::R, double>::value, "exact-sum stencil is FP64 only");
  const int F = acc.fixF(), eadj = f.F - F;
  const longlong2 cc = acc.fx0();
  bool bad = fbad(cc);
  long long s1x = 0, s1y = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const longlong2 u = acc.fx1(k, 1), w = acc.fx1(k, -1);
    bad |= fbad(u) | fbad(w);
    s1x += u.x + w.x;
    s1y += u.y + w.y;
  }
  const double Nc = Ng * f.cLF;   // physical N_c, for the walls' ghosts and the fallback
  if constexpr (ORDER == 2) {
    if (bad) {
      const double2 aL = a_lap_slow<T, D, ORDER>(f, acc, idx, c, pc, Nc);
      return {aL.x * f.invcLF, aL.y * f.invcLF};
    }
    return {i2d_rn(s1x - 2 * D * cc.x, eadj), i2d_rn(s1y - 2 * D * cc.y, eadj)};
  }
  const bool wall = near_wall2<D>(idx, f.n);
  long long s2x = 0, s2y = 0;
  if (!wall) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const longlong2 lo = acc.fx1(k, -2), hi = acc.fx1(k, 2);
      bad |= fbad(lo) | fbad(hi);
      s2x += lo.x + hi.x;
      s2y += lo.y + hi.y;
    }
  } else {
    // h^2 D_c from the exact face-neighbour sum (the MSD ghosts' ratio term needs it)
    const double2 dh = {i2d_rn(s1x - 2 * D * cc.x, -F), i2d_rn(s1y - 2 * D * cc.y, -F)};
    const longlong2 s2 = exact_s2_wall<T, D>(f, acc, idx, c, pc, dh, Nc, m2, F, &bad);
    s2x = s2.x;
    s2y = s2.y;
  }
  if (bad) {
    const double2 aL = a_lap_slow<T, D, ORDER>(f, acc, idx, c, pc, Nc);
    return {aL.x * f.invcLF, aL.y * f.invcLF};
  }
  const long long Sx = 16 * s1x - s2x - 30 * D * cc.x;
  const long long Sy = 16 * s1y - s2y - 30 * D * cc.y;
  return {i2d_rn(Sx, eadj), i2d_rn(Sy, eadj)};
}

// The exact-sum Laplacian at a deep-interior site (no wall within two cells),
// in units of cLF like a_lap_exact, without its wall branch.
template <class T, int D, int ORDER, class Acc>
__device__ __forceinline__ double2 a_lap_exact_deep(const Field<T>& f, const Acc& acc, const int* idx, int64_t c,
                                                    double2 pc, double Ng) {
  const int eadj = f.F - acc.fixF();
  const longlong2 cc = acc.fx0();
  bool bad = fbad(cc);
  long long s1x = 0, s1y = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const longlong2 u = acc.fx1(k, 1), w = acc.fx1(k, -1);
    bad |= fbad(u) | fbad(w);
    s1x += u.x + w.x;
    s1y += u.y + w.y;
  }
  // out-of-range fallback: the FP64 stencil without the wall branch (no wall is within reach of a deep
  // site, and a periodic grid has none)
  if constexpr (ORDER == 2) {
    if (bad) {
      const double2 aL = a_lap_body<T, D, ORDER, Acc, false>(f, acc, idx, c, pc, Ng * f.cLF);
      return {aL.x * f.invcLF, aL.y * f.invcLF};
    }
    return {i2d_rn(s1x - 2 * D * cc.x, eadj), i2d_rn(s1y - 2 * D * cc.y, eadj)};
  }
  long long s2x = 0, s2y = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const longlong2 lo = acc.fx1(k, -2), hi = acc.fx1(k, 2);
    bad |= fbad(lo) | fbad(hi);
    s2x += lo.x + hi.x;
    s2y += lo.y + hi.y;
  }
  if (bad) {
    const double2 aL = a_lap_body<T, D, ORDER, Acc, false>(f, acc, idx, c, pc, Ng * f.cLF);
    return {aL.x * f.invcLF, aL.y * f.invcLF};
  }
  const long long Sx = 16 * s1x - s2x - 30 * D * cc.x;
  const long long Sy = 16 * s1y - s2y - 30 * D * cc.y;
  return {i2d_rn(Sx, eadj), i2d_rn(Sy, eadj)};
}

template <class T, int D>
__device__ __forceinline__ longlong2 GAcc<T, D>::fx0() const { return fix2(ld2<double>(f.in, c), cur_fix(f)); }
template <class T, int D>
__device__ __forceinline__ longlong2 GAcc<T, D>::fx1(int k, int s) const {
  return fix2(ld2<double>(f.in, c + s * f.st[k]), cur_fix(f));
}
template <class T, int D>
__device__ __forceinline__ longlong2 GAcc<T, D>::fx2(int k, int s, int j, int t) const {
  return fix2(ld2<double>(f.in, c + s * f.st[k] + t * f.st[j]), cur_fix(f));
}

// Everything a stage writes, on top of the field it reads.
template <class T>
struct StageArgs {
  Field<T> f;
  const typename T::C* psin;   // Psi^n in stage precision (stage 1: == f.in)
  typename T::C* ktot;         // K_tot
  typename T::C* out;          // Psi_tmp / Psi_out (stages 1-3); F (stage 0)
  typename T::M* master;       // where stage 4 writes the master Psi^{n+1}
  const typename T::M* master_in;   // where stage 4 reads the master Psi^n (== master when updated in place)
  typename T::C* n32;          // PMix: FP32 copy of Psi^{n+1} written in stage 4
  typename T::R dtc;           // dt/2, dt/2, dt, dt/6 for stages 1..4
  double dt6;                  // dt/6 in FP64 (PMix stage 4)
  int stage;                   // 0 = write F only, 1..4 = RK4 stage
  unsigned int* flag;          // bit 0: non-finite Psi
  const typename T::VR* Vs;    // exact-sum stages: V / cLF (nullptr when V is)
  unsigned int* emax;          // exact-sum stage 4: device word that collects the largest biased exponent of
                               //   the components of Psi^{n+1} (nullptr otherwise)
  int xwall;                   // 3D tiled path: the shell also owns x in [2, 1 + xwall] and its mirror
                               // (deep-interior kernels start at x = 2 + xwall); 0 by default
};

// float <-> double on the integer pipe (GB300 issues FP64-pipe instructions,
// conversions included, at 1/75 of the FP32 rate).  Both follow IEEE-754:
// widening is exact, narrowing rounds to nearest even; zeros, subnormals,
// infinities and NaN take the hardware conversion.
__device__ __forceinline__ double f2d_exact(float v) {
  const unsigned int u = __float_as_uint(v);
  const unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return double(v);
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                  ((unsigned long long)(e - 127u + 1023u) << 52) |
                                  ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ float d2f_rn(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int e = int((u >> 52) & 0x7FF) - 1023 + 127;   // biased float exponent
  if (e <= 0 || e >= 0xFF) return float(v);             // float subnormal/zero, overflow, Inf, NaN
  const unsigned int sgn = (unsigned int)(u >> 32) & 0x80000000u;
  const unsigned long long m = u & 0x000FFFFFFFFFFFFFull;
  unsigned int mf = (unsigned int)(m >> 29);
  const unsigned long long rem = m & 0x1FFFFFFFull, half = 0x10000000ull;
  unsigned int ef = (unsigned int)e;
  if (rem > half || (rem == half && (mf & 1u))) {
    if (++mf == 0x800000u) { mf = 0; ++ef; }
    if (ef >= 0xFFu) return float(v);                   // rounds up to overflow
  }
  return __uint_as_float(sgn | (ef << 23) | mf);
}

// isfinite by the exponent bits (integer pipe; the FP64 pipe is GB300's scarcest unit)
__device__ __forceinline__ bool finite_bits(double v) {
  return (__double2hiint(v) & 0x7FF00000) != 0x7FF00000;
}
__device__ __forceinline__ bool finite_bits(float v) { return (__float_as_uint(v) & 0x7F800000u) != 0x7F800000u; }

// The pointwise operands of one site's update, loaded ahead of use.
template <class T>
struct PointVals {
  typename T::R v;      // V at the site
  typename T::C pn;     // Psi^n (stage precision), stages 1-3
  typename T::C K;      // K_tot, stages 2-4
  typename T::M mst;    // master Psi^n, stage 4
};

// S = the stage when known at compile time, -1 = read A.stage.  G: the
// exact-sum stages, which read the scaled potential V / cLF (see rk_apply).
template <class T, int S = -1, bool G = false>
__device__ __forceinline__ PointVals<T> load_point(const StageArgs<T>& A, int64_t i, bool with_v) {
  PointVals<T> p;
  const int st = (S >= 0) ? S : A.stage;
  p.v = with_v ? ldv<typename T::R>(G ? A.Vs : A.f.V, i) : typename T::R(0);
  if (st >= 1 && st <= 3) p.pn = A.psin[i];
  if (st >= 2) p.K = A.ktot[i];
  if (st == 4) p.mst = A.master_in[i];
  return p;
}

// Apply stage A.stage of Eq. RK4_GPU at site i with k = F.
// Returns, for stage 4, the largest biased exponent of the components written
// to the FP64 master (0 otherwise; see StageArgs::emax).
template <class T, int S = -1>
__device__ __forceinline__ unsigned int rk_apply(const StageArgs<T>& A, int64_t i, typename V2<typename T::R>::t F,
                                                 const PointVals<T>& p) {
  using R = typename T::R;
  using C = typename T::C;
  switch ((S >= 0) ? S : A.stage) {
    case 0:  // F itself: dtc = 1, or cLF for the exact-sum stages (whose F is in units of cLF)
      A.out[i] = C{A.dtc * F.x, A.dtc * F.y};
      break;
    case 1:  // K_tot = k; Psi_tmp = Psi^n + (dt/2) k
      A.ktot[i] = C{F.x, F.y};
      A.out[i] = C{fma(A.dtc, F.x, p.pn.x), fma(A.dtc, F.y, p.pn.y)};
      break;
    case 2:
    case 3:  // K_tot += 2k; Psi_out = Psi^n + (dt/2) k  |  Psi_tmp = Psi^n + dt k
      A.ktot[i] = C{fma(R(2), F.x, p.K.x), fma(R(2), F.y, p.K.y)};
      A.out[i] = C{fma(A.dtc, F.x, p.pn.x), fma(A.dtc, F.y, p.pn.y)};
      break;
    default: {  // Psi^{n+1} = Psi^n + (dt/6)(K_tot + k)
      typename T::M q;
      if constexpr (std::is_same<typename T::M, C>::value) {
        q.x = fma(A.dtc, p.K.x + F.x, p.mst.x);
        q.y = fma(A.dtc, p.K.y + F.y, p.mst.y);
      } else {  // FP64 accumulator over FP32 stages: the FP32 increment added to the FP64 master
        const float ix = A.dtc * (p.K.x + F.x), iy = A.dtc * (p.K.y + F.y);
        q.x = p.mst.x + f2d_exact(ix);
        q.y = p.mst.y + f2d_exact(iy);
        A.n32[i] = C{d2f_rn(q.x), d2f_rn(q.y)};
      }
      A.master[i] = q;
      if (!(finite_bits(q.x) && finite_bits(q.y))) atomicOr(A.flag, 1u);
      return max(expo_bits(q.x), expo_bits(q.y));
    }
  }
  return 0u;
}

template <class T, int S = -1>
__device__ __forceinline__ unsigned int rk_update(const StageArgs<T>& A, int64_t i, typename V2<typename T::R>::t F) {
  return rk_apply<T, S>(A, i, F, load_point<T, S>(A, i, false));
}

// Update every boundary site whose b-1 neighbour is the interior site c
// (c + sum_k o_k e_k with o_k in {0} u {-1 if idx==1} u {+1 if idx==n-2}, not
// all 0), with F_b = 0 (Dirichlet), F_b = i Im(F_c / Psi_c) Psi_b (MSD) or
// F_b = i N_b Psi_b (L0; in units of cLF on the exact-sum stages, like F_c).
// Out of line: only sites next to a wall call it.
// S: the RK4 stage when the caller's kernel is built for one (-1: A.stage at run time).
template <class T, int D, bool EXACT, class Acc, int S = -1>
__device__ __forceinline__ unsigned int serve_walls(const StageArgs<T>& A, const Acc& acc, const int* idx, int64_t c,
                                                 typename V2<typename T::R>::t pc, typename V2<typename T::R>::t F,
                                                 typename T::R m2w) {
  using R = typename T::R;
  using C2 = typename V2<R>::t;
  const Field<T>& f = A.f;
  R theta = R(0);
  unsigned int ex = 0;
  if (f.bc == BC_MSD) {
    // Im(F_c / Psi_c) = Im(F_c conj(Psi_c)) / |Psi_c|^2, 0 below the guard; the exact-sum stages pass
    // |Psi_c|^2 in (m2w, already guarded), shared with the site's ghosts
    const R m2 = EXACT ? m2w : norm2(pc);
    if (EXACT ? m2 > R(0) : m2 > f.tiny) theta = fma(F.y, pc.x, -(F.x * pc.y)) / m2;
  }
  // all offsets o in {-1, 0, 1}^D except 0, where -1 needs idx == 1 and +1 needs idx == n - 2: per axis
  // the options {0, -1 if idx == 1, +1 if idx == n - 2}, walked as a mixed-radix counter in a loop that
  // is not unrolled, so the boundary-site update below is emitted once (a face site has one such
  // neighbour, an edge three, a corner seven); each boundary site is updated on its own, so the order
  // of the walk does not change any result
  int opt[D][3], cnt[D], total = 1;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    cnt[k] = 1;
    opt[k][0] = 0;
    if (idx[k] == 1) opt[k][cnt[k]++] = -1;
    if (idx[k] == f.n[k] - 2) opt[k][cnt[k]++] = 1;
    total *= cnt[k];
  }
#pragma unroll 1
  for (int q = 1; q < total; ++q) {
    int o[D];
    int r = q;
    int64_t b = c;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
      const int ck = cnt[k];
      const int v = r % ck;
      r /= ck;
      o[k] = v == 0 ? 0 : (v == 1 ? opt[k][1] : opt[k][2]);
      b += o[k] * f.st[k];
    }
    C2 Fb = {R(0), R(0)};
    if (f.bc == BC_MSD) {
      const C2 pb = acc.atv(o);
      Fb = {-theta * pb.y, theta * pb.x};
    } else if (f.bc == BC_L0) {
      const C2 pb = acc.atv(o);
      const R Nb = fma(EXACT ? f.sG : f.s, norm2(pb), -ldv<R>(EXACT ? A.Vs : f.V, b));
      Fb = {-Nb * pb.y, Nb * pb.x};
    }
    ex = max(ex, rk_update<T, S>(A, b, Fb));
  }
  return ex;
}

// The full per-site work: F at interior site c, its update, and the update of
// every boundary site whose b-1 neighbour is c.  `p` holds c's pointwise
// operands (load_point).
template <class T, int D, int ORDER, bool EXACT, class Acc, int S = -1>
__device__ __forceinline__ unsigned int process_site_pv(const StageArgs<T>& A, const Acc& acc, const int* idx,
                                                        int64_t c, const PointVals<T>& p) {
  using R = typename T::R;
  using C2 = typename V2<R>::t;
  const Field<T>& f = A.f;
  const C2 pc = acc.at0();
  // exact-sum stages work in units of cLF: Nc / cLF (p.v holds V / cLF there)
  const R Nc = fma(EXACT ? f.sG : f.s, norm2(pc), -p.v);
  R m2w = R(0);
  if constexpr (EXACT) {   // |Psi_c|^2 of an MSD wall-adjacent site (0 below the guard), for its ghosts and theta
    if (f.bc == BC_MSD && near_wall2<D>(idx, f.n)) {
      const R m2 = norm2(pc);
      m2w = (m2 > f.tiny) ? m2 : R(0);
    }
  }
  C2 aL;
  if constexpr (EXACT) aL = a_lap_exact<T, D, ORDER>(f, acc, idx, c, pc, Nc, m2w);
  else aL = a_lap<T, D, ORDER>(f, acc, idx, c, pc, Nc);
  const C2 F = {-fma(Nc, pc.y, aL.y), fma(Nc, pc.x, aL.x)};
  unsigned int ex = rk_apply<T, S>(A, c, F, p);

  bool near = false;
#pragma unroll
  for (int k = 0; k < D; ++k) near |= (idx[k] == 1) | (idx[k] == f.n[k] - 2);
  if (near) ex = max(ex, serve_walls<T, D, EXACT, Acc, S>(A, acc, idx, c, pc, F, m2w));
  return ex;
}

template <class T, int D, int ORDER, bool EXACT, class Acc, int S = -1>
__device__ __forceinline__ unsigned int process_site(const StageArgs<T>& A, const Acc& acc, const int* idx,
                                                     int64_t c) {
  return process_site_pv<T, D, ORDER, EXACT, Acc, S>(A, acc, idx, c, load_point<T, S, EXACT>(A, c, true));
}

// ---------------------------------------------------------------------------
// Periodic grids (BC_PERIODIC; the boundary the stability analysis of Sec.
// 3.4 assumes): there are no boundary sites, every site is updated, and the
// site N[k] along axis k is site 0 again.  Every face neighbour of every site
// is then an ordinary site, so 2SHOC is the five-point form everywhere (the
// identity above needs no wall ghosts).
// ---------------------------------------------------------------------------
template <class T, int D>
struct GAccP {
  using R = typename T::R;
  using C2 = typename V2<R>::t;
  const Field<T>& f;
  int64_t c;
  int idx[D];
  __device__ __forceinline__ GAccP(const Field<T>& f_, int64_t c_, const int* idx_) : f(f_), c(c_) {
#pragma unroll
    for (int k = 0; k < D; ++k) idx[k] = idx_[k];
  }
  // stride offset of s cells (|s| <= 2) along axis k, wrapped into [0, N[k])
  __device__ __forceinline__ int64_t sh(int k, int s) const {
    int i = idx[k] + s;
    i = i < 0 ? i + f.n[k] : (i >= f.n[k] ? i - f.n[k] : i);
    return (int64_t)(i - idx[k]) * f.st[k];
  }
  __device__ __forceinline__ C2 at0() const { return ld2<R>(f.in, c); }
  __device__ __forceinline__ C2 at1(int k, int s) const { return ld2<R>(f.in, c + sh(k, s)); }
  __device__ __forceinline__ C2 at2(int k, int s, int j, int t) const { return ld2<R>(f.in, c + sh(k, s) + sh(j, t)); }
  __device__ __forceinline__ longlong2 fx0() const { return fix2(ld2<double>(f.in, c), cur_fix(f)); }
  __device__ __forceinline__ longlong2 fx1(int k, int s) const {
    return fix2(ld2<double>(f.in, c + sh(k, s)), cur_fix(f));
  }
  __device__ __forceinline__ int fixF() const { return cur_fix(f); }
};

// F and the stage update at site c (multi-index idx) of a periodic grid, the
// operands from an accessor whose neighbours wrap.
template <class T, int D, int ORDER, bool EXACT, class Acc>
__device__ __forceinline__ unsigned int process_site_periodic_acc(const StageArgs<T>& A, const Acc& acc,
                                                                  const int* idx, int64_t c) {
  using R = typename T::R;
  using C2 = typename V2<R>::t;
  const Field<T>& f = A.f;
  const PointVals<T> p = load_point<T, -1, EXACT>(A, c, true);
  const C2 pc = acc.at0();
  const R Nc = fma(EXACT ? f.sG : f.s, norm2(pc), -p.v);   // units of cLF on the exact-sum stages
  C2 aL;
  if constexpr (EXACT) aL = a_lap_exact_deep<T, D, ORDER>(f, acc, idx, c, pc, Nc);
  else aL = a_lap_body<T, D, ORDER, Acc, false>(f, acc, idx, c, pc, Nc);
  return rk_apply<T>(A, c, {-fma(Nc, pc.y, aL.y), fma(Nc, pc.x, aL.x)}, p);
}

template <class T, int D, int ORDER, bool EXACT>
__device__ __forceinline__ unsigned int process_site_periodic(const StageArgs<T>& A, const int* idx, int64_t c) {
  return process_site_periodic_acc<T, D, ORDER, EXACT>(A, GAccP<T, D>(A.f, c, idx), idx, c);
}

// How a stage is launched: kernel variant, CTA tile, and (3D tiled kernel)
// the TMA descriptor of the stage input when the layout allows TMA.
struct LaunchCfg {
  int variant;
  int tile_cfg;
  const void* tmap;        // CUtensorMap* of A.f.in for the tile's box, or nullptr
  long long spin_limit;    // bound on any device-side wait, in SM clock cycles
  unsigned int extra_tx;   // test hook: extra bytes every TMA barrier waits for (0 in normal use)
  cudaStream_t side;       // if set, the wall-shell kernel runs on this stream, concurrently with the
  cudaEvent_t ev_fork;     //   deep-interior kernel (fork after ev_fork on the main stream, join on ev_join)
  cudaEvent_t ev_join;
  cudaStream_t side_yx[2];   // if set (3D), the y- and x-wall slabs run on these streams, concurrently with
  cudaEvent_t ev_join_yx[2]; //   the z-wall slab on `side` and the deep kernel (joined on ev_join_yx)
                             //   (shell launchers that use one stream leave them idle: fork and join only)
};

// Launch the deep-interior part and the wall-shell part of one stage; with a
// side stream they run concurrently (they write disjoint sites and read the
// same stage input).
template <class DeepFn, class ShellFn>
cudaError_t launch_deep_and_shell(const LaunchCfg& L, cudaStream_t stream, bool deep, DeepFn&& run_deep,
                                  ShellFn&& run_shell) {
  cudaError_t e = cudaSuccess;
  if (L.side && deep) {
    // With the three wall streams (3D) the deep kernel is issued first: its CTAs take the SMs and the
    // three slabs, all in flight at once, fill the slots its last wave leaves (measured on 256x256x512:
    // 1-4 % faster steps than the slabs issued first on one stream; issuing the deep kernel first
    // without the extra streams was slower in FP64).
    const int nx = L.side_yx[0] ? 2 : 0;
    const bool deep_first = nx > 0;
    if ((e = cudaEventRecord(L.ev_fork, stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(L.side, L.ev_fork, 0)) != cudaSuccess) return e;
    for (int i = 0; i < nx; ++i)
      if ((e = cudaStreamWaitEvent(L.side_yx[i], L.ev_fork, 0)) != cudaSuccess) return e;
    if (deep_first && (e = run_deep(stream)) != cudaSuccess) return e;
    if ((e = run_shell(L.side)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(L.ev_join, L.side)) != cudaSuccess) return e;
    for (int i = 0; i < nx; ++i)
      if ((e = cudaEventRecord(L.ev_join_yx[i], L.side_yx[i])) != cudaSuccess) return e;
    if (!deep_first && (e = run_deep(stream)) != cudaSuccess) return e;
    for (int i = 0; i < nx; ++i)
      if ((e = cudaStreamWaitEvent(stream, L.ev_join_yx[i], 0)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(stream, L.ev_join, 0);
  }
  if (deep && (e = run_deep(stream)) != cudaSuccess) return e;
  return run_shell(stream);
}

// Host-visible launch entry points (defined in stage_*.cu).
template <class T, int D, int ORDER>
cudaError_t launch_stage(const StageArgs<T>& A, const LaunchCfg& L, cudaStream_t stream);

}  // namespace nlse
