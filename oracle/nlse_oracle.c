/*
 * Plain FP64 CPU oracle for the NLSEmagic RK4 integrator (arXiv 1203.1263).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load this file's library.  It shares no
 * code, header, table or helper with the CUDA library; the two meet only in
 * the seeded input arrays.
 *
 * It computes the method the slow, obvious way, one whole-grid array per
 * quantity, in the order the paper states it:
 *
 *   F(Psi) = i [ a Lap(Psi) + (s|Psi|^2 - V) Psi ]                (Sec. 3.1)
 *   split into real and imaginary parts as in Sec. 5.2, Eq. fsplit.
 *
 *   Lap: order 2 = central difference (Sec. 3.2, step 1 of Eqs. 2shoc1d,
 *        2d2shocs1, 3d2shocs); order 4 = the two-step compact 2SHOC scheme
 *        (Eqs. 2shoc1d2, 2d2shocs2, 3d2shocs2).  The 3D step-2 tables are read
 *        as the planes j+1, j, j-1: D has 6 face neighbours with weight 1 and
 *        centre -10, Psi has the 12 edge-diagonal neighbours with weight 1 and
 *        centre -12.
 *
 *   Boundary (Sec. 3.3): a site is a boundary site when any of its indices is
 *   0 or N-1.  Its "b-1" neighbour steps one cell inward along every axis on
 *   which it is a boundary index (the nearest interior site).
 *     Dirichlet: dPsi_b/dt = 0 (Eq. BCDdt);
 *                Laplacian form D_b = -(1/a)(s|Psi_b|^2 - V_b) Psi_b (Eq. BCDlap).
 *     MSD:       dPsi_b/dt = i Im[F_{b-1}/Psi_{b-1}] Psi_b (Eq. msd);
 *                D_b = [Re(D_{b-1}/Psi_{b-1}) + (N_{b-1} - N_b)/a] Psi_b
 *                (Eq. BCMSDlap with Im(i z) = Re(z) and the CD value D_{b-1}),
 *                N = s|Psi|^2 - V.  When |Psi_{b-1}|^2 <= 1e-300 the ratio
 *                term is taken as 0.
 *     L0:        dPsi_b/dt = i (s|Psi_b|^2 - V_b) Psi_b (Eq. BCL0dt);
 *                D_b = 0 (Eq. BCL0lap).
 *     The boundary D_b enters only the 2SHOC step 2 of interior sites.
 *   Periodic (not one of the paper's boundary forms; its stability analysis,
 *   Sec. 3.4, assumes it): the grid has no boundary sites.  Site N[k] along
 *   axis k is site 0 again (period N[k] h), so every site is interior and
 *   every neighbour index is taken modulo N[k].
 *
 *   RK4: the ten-step algorithmic form of Sec. 3.1, Eq. RK4, with
 *   K_tot, Psi_tmp and K_tmp held as whole-grid arrays.
 *
 *   Mass   M = h^d sum_{all sites} |Psi|^2.
 *   Energy E = h^d sum_{interior} [ -a Re(conj(Psi) Lap Psi) + V|Psi|^2 - (s/2)|Psi|^4 ]
 *   with the scheme's own Laplacian (same order and boundary D_b).
 *   Both sums use Neumaier's compensated summation (Neumaier 1974).
 *
 * Layout: C order (last index fastest); psi is interleaved (re, im) doubles;
 * V is real with the same shape, or NULL for V = 0.
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define BC_DIRICHLET 0
#define BC_MSD 1
#define BC_L0 2
#define BC_PERIODIC 3
#define MSD_TINY 1e-300

typedef struct {
  int d;               /* 1, 2 or 3 */
  int64_t n[3];        /* extents, n[d-1] is the fastest axis */
  int64_t st[3];       /* strides in sites */
  int64_t total;
  double h, a, s;
  const double *V;     /* may be NULL */
  int bc, order;
} grid;

static int setup(grid *g, int d, const int64_t *n, double h, double a, double s, const double *V, int bc,
                 int order) {
  if (d < 1 || d > 3) return -1;
  g->d = d;
  g->total = 1;
  for (int k = 0; k < 3; ++k) { g->n[k] = 1; g->st[k] = 0; }
  for (int k = d - 1; k >= 0; --k) {
    if (n[k] < 3) return -1;
    g->n[k] = n[k];
    g->st[k] = g->total;
    g->total *= n[k];
  }
  g->h = h; g->a = a; g->s = s; g->V = V; g->bc = bc; g->order = order;
  if (!(order == 2 || order == 4)) return -1;
  if (!(bc == BC_DIRICHLET || bc == BC_MSD || bc == BC_L0 || bc == BC_PERIODIC)) return -1;
  return 0;
}

static void decode(const grid *g, int64_t p, int64_t idx[3]) {
  for (int k = 0; k < g->d; ++k) idx[k] = (p / g->st[k]) % g->n[k];
}

static int is_boundary(const grid *g, int64_t p) {
  int64_t idx[3];
  if (g->bc == BC_PERIODIC) return 0;
  decode(g, p, idx);
  for (int k = 0; k < g->d; ++k)
    if (idx[k] == 0 || idx[k] == g->n[k] - 1) return 1;
  return 0;
}

/* b-1: one step inward along every axis on which p is a boundary index. */
static int64_t inward(const grid *g, int64_t p) {
  int64_t idx[3], q = p;
  decode(g, p, idx);
  for (int k = 0; k < g->d; ++k) {
    if (idx[k] == 0) q += g->st[k];
    else if (idx[k] == g->n[k] - 1) q -= g->st[k];
  }
  return q;
}

/* The site o = (o0, o1, o2) cells away from p (o_k along axis k).  On a
 * periodic grid each index wraps modulo N[k]; otherwise the caller only asks
 * for sites inside the grid (interior p, |o_k| <= 1). */
static int64_t nb(const grid *g, int64_t p, int o0, int o1, int o2) {
  const int o[3] = {o0, o1, o2};
  if (g->bc != BC_PERIODIC) return p + o0 * g->st[0] + o1 * g->st[1] + o2 * g->st[2];
  int64_t idx[3], q = 0;
  decode(g, p, idx);
  for (int k = 0; k < g->d; ++k) q += ((idx[k] + o[k] + g->n[k]) % g->n[k]) * g->st[k];
  return q;
}

/* the site one cell away from p along axis k, in direction s (+1 or -1) */
static int64_t nb1(const grid *g, int64_t p, int k, int s) {
  return nb(g, p, k == 0 ? s : 0, k == 1 ? s : 0, k == 2 ? s : 0);
}

static double Vat(const grid *g, int64_t p) { return g->V ? g->V[p] : 0.0; }

/* N = s|Psi|^2 - V */
static double Nat(const grid *g, const double *psi, int64_t p) {
  double re = psi[2 * p], im = psi[2 * p + 1];
  return g->s * (re * re + im * im) - Vat(g, p);
}

/* ---- Step 1: central-difference D (Eqs. 2shoc1d, 2d2shocs1, 3d2shocs) ---- */
/* interior sites: (1/h^2) (sum over the 2d face neighbours - 2d Psi) */
static void compute_D_interior(const grid *g, const double *psi, double *D) {
  const double inv_h2 = 1.0 / (g->h * g->h);
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < g->total; ++p) {
    if (is_boundary(g, p)) { D[2 * p] = D[2 * p + 1] = 0.0; continue; }
    for (int c = 0; c < 2; ++c) {
      double sum = 0.0;
      for (int k = 0; k < g->d; ++k) sum += psi[2 * nb1(g, p, k, 1) + c] + psi[2 * nb1(g, p, k, -1) + c];
      sum += -2.0 * g->d * psi[2 * p + c];
      D[2 * p + c] = inv_h2 * sum;
    }
  }
}

/* boundary sites: the Laplacian forms of the boundary conditions,
 * Eqs. BCDlap (Dirichlet), BCMSDlap (MSD) and BCL0lap (L0).  Needs the
 * interior D first. */
static void compute_D_boundary(const grid *g, const double *psi, double *D) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < g->total; ++p) {
    if (!is_boundary(g, p)) continue;
    const double re = psi[2 * p], im = psi[2 * p + 1];
    if (g->bc == BC_DIRICHLET) {
      const double f = -(1.0 / g->a) * Nat(g, psi, p);
      D[2 * p] = f * re;
      D[2 * p + 1] = f * im;
    } else if (g->bc == BC_L0) {
      D[2 * p] = 0.0;
      D[2 * p + 1] = 0.0;
    } else {
      const int64_t q = inward(g, p);
      const double qr = psi[2 * q], qi = psi[2 * q + 1];
      const double m2 = qr * qr + qi * qi;
      double ratio_re = 0.0; /* Re(D_q / Psi_q) */
      if (m2 > MSD_TINY) ratio_re = (D[2 * q] * qr + D[2 * q + 1] * qi) / m2;
      const double f = ratio_re + (Nat(g, psi, q) - Nat(g, psi, p)) / g->a;
      D[2 * p] = f * re;
      D[2 * p + 1] = f * im;
    }
  }
}

/* D at every site: interior CD values, and for 2SHOC the boundary forms. */
static void compute_D(const grid *g, const double *psi, double *D) {
  compute_D_interior(g, psi, D);
  if (g->order == 4) compute_D_boundary(g, psi, D);
}

/* ---- Step 2: the Laplacian at interior sites ---- */
static void compute_L(const grid *g, const double *psi, const double *D, double *L) {
  const double inv_h2 = 1.0 / (g->h * g->h);
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < g->total; ++p) {
    if (is_boundary(g, p)) { L[2 * p] = L[2 * p + 1] = 0.0; continue; }
    for (int c = 0; c < 2; ++c) {
/* Psi and D at the site (o0, o1, o2) cells away from p */
#define PS(o0, o1, o2) psi[2 * nb(g, p, o0, o1, o2) + c]
#define DD(o0, o1, o2) D[2 * nb(g, p, o0, o1, o2) + c]
      double v;
      if (g->order == 2) {
        v = DD(0, 0, 0);
      } else if (g->d == 1) {
        /* Eq. 2shoc1d2: (7/6) D_i - (1/12)(D_{i+1} + D_{i-1}) */
        v = (7.0 / 6.0) * DD(0, 0, 0) - (1.0 / 12.0) * (DD(1, 0, 0) + DD(-1, 0, 0));
      } else if (g->d == 2) {
        /* Eq. 2d2shocs2: -(1/12)[plus stencil, centre -12] D + (1/(6h^2))[corners 1, centre -4] Psi */
        double sd = DD(1, 0, 0) + DD(-1, 0, 0) + DD(0, 1, 0) + DD(0, -1, 0) - 12.0 * DD(0, 0, 0);
        double sp = PS(1, 1, 0) + PS(1, -1, 0) + PS(-1, 1, 0) + PS(-1, -1, 0) - 4.0 * PS(0, 0, 0);
        v = -(1.0 / 12.0) * sd + (inv_h2 / 6.0) * sp;
      } else {
        /* Eq. 3d2shocs2: -(1/12)[6 face neighbours, centre -10] D
         *                + (1/(6h^2))[12 edge-diagonal neighbours, centre -12] Psi */
        double sd = DD(1, 0, 0) + DD(-1, 0, 0) + DD(0, 1, 0) + DD(0, -1, 0) + DD(0, 0, 1) + DD(0, 0, -1) -
                    10.0 * DD(0, 0, 0);
        double sp = 0.0;
        /* plane j+1 and j-1 (axis 0 = j here): the four in-plane face neighbours */
        sp += PS(1, 1, 0) + PS(1, -1, 0) + PS(1, 0, 1) + PS(1, 0, -1);
        sp += PS(-1, 1, 0) + PS(-1, -1, 0) + PS(-1, 0, 1) + PS(-1, 0, -1);
        /* plane j: the four corners */
        sp += PS(0, 1, 1) + PS(0, 1, -1) + PS(0, -1, 1) + PS(0, -1, -1);
        sp += -12.0 * PS(0, 0, 0);
        v = -(1.0 / 12.0) * sd + (inv_h2 / 6.0) * sp;
      }
      L[2 * p + c] = v;
#undef PS
#undef DD
    }
  }
}

/* F(Psi) into F (whole grid).  Scratch D and L are whole-grid arrays. */
static void evalF(const grid *g, const double *psi, double *F, double *D, double *L) {
  compute_D(g, psi, D);
  compute_L(g, psi, D, L);
  /* Step 3: interior sites, Eq. fsplit */
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < g->total; ++p) {
    if (is_boundary(g, p)) continue;
    const double re = psi[2 * p], im = psi[2 * p + 1];
    const double m2 = re * re + im * im, v = Vat(g, p);
    F[2 * p] = -g->a * L[2 * p + 1] - g->s * m2 * im + v * im;
    F[2 * p + 1] = g->a * L[2 * p] + g->s * m2 * re - v * re;
  }
  /* Step 4: boundary sites, Eqs. BCDdt / msd / BCL0dt */
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < g->total; ++p) {
    if (!is_boundary(g, p)) continue;
    if (g->bc == BC_DIRICHLET) {
      F[2 * p] = 0.0;
      F[2 * p + 1] = 0.0;
    } else if (g->bc == BC_L0) {
      /* i N_b Psi_b */
      const double nb = Nat(g, psi, p);
      F[2 * p] = -nb * psi[2 * p + 1];
      F[2 * p + 1] = nb * psi[2 * p];
    } else {
      const int64_t q = inward(g, p);
      const double qr = psi[2 * q], qi = psi[2 * q + 1];
      const double m2 = qr * qr + qi * qi;
      double theta = 0.0; /* Im(F_q / Psi_q) */
      if (m2 > MSD_TINY) theta = (F[2 * q + 1] * qr - F[2 * q] * qi) / m2;
      /* i theta Psi_b */
      F[2 * p] = -theta * psi[2 * p + 1];
      F[2 * p + 1] = theta * psi[2 * p];
    }
  }
}

/* ---------------------------------------------------------------------------
 * Exported entry points (ctypes).  All return 0 on success, -1 on bad
 * arguments, -2 when scratch memory could not be allocated.
 * ------------------------------------------------------------------------- */

int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* F(Psi) for the whole grid (Sec. 3.1 with the Sec. 3.3 boundary forms). */
int oracle_evalF(int d, const int64_t *n, double h, double a, double s, const double *V, int bc, int order,
                 const double *psi, double *F) {
  grid g;
  if (setup(&g, d, n, h, a, s, V, bc, order)) return -1;
  double *D = calloc(2 * g.total, sizeof(double)), *L = calloc(2 * g.total, sizeof(double));
  if (!D || !L) { free(D); free(L); return -2; }
  evalF(&g, psi, F, D, L);
  free(D); free(L);
  return 0;
}

/* Step 1 (D, with the boundary Laplacian forms) and step 2 (Lap at interior
 * sites; 0 at boundary sites) separately, for the stencil tests. */
int oracle_laplacian(int d, const int64_t *n, double h, double a, double s, const double *V, int bc, int order,
                     const double *psi, double *D, double *L) {
  grid g;
  if (setup(&g, d, n, h, a, s, V, bc, order)) return -1;
  compute_D(&g, psi, D);
  compute_L(&g, psi, D, L);
  return 0;
}

/* nsteps RK4 steps of size dt on psi in place, Sec. 3.1 Eq. RK4, steps 1-10. */
int oracle_rk4(int d, const int64_t *n, double h, double a, double s, const double *V, int bc, int order,
               double dt, int64_t nsteps, double *psi) {
  grid g;
  if (setup(&g, d, n, h, a, s, V, bc, order)) return -1;
  const int64_t m = 2 * g.total;
  double *Ktot = malloc(m * sizeof(double)), *Ptmp = malloc(m * sizeof(double)),
         *Ktmp = malloc(m * sizeof(double)), *D = calloc(m, sizeof(double)), *L = calloc(m, sizeof(double));
  if (!Ktot || !Ptmp || !Ktmp || !D || !L) {
    free(Ktot); free(Ptmp); free(Ktmp); free(D); free(L);
    return -2;
  }
  const double half = dt / 2.0, sixth = dt / 6.0;
  for (int64_t step = 0; step < nsteps; ++step) {
    evalF(&g, psi, Ktot, D, L);                                   /* 1) K_tot = F(Psi^n) */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) Ptmp[i] = psi[i] + half * Ktot[i];   /* 2) */
    evalF(&g, Ptmp, Ktmp, D, L);                                  /* 3) K_tmp = F(Psi_tmp) */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
      Ktot[i] = Ktot[i] + 2.0 * Ktmp[i];                          /* 4) */
      Ptmp[i] = psi[i] + half * Ktmp[i];                          /* 5) */
    }
    evalF(&g, Ptmp, Ktmp, D, L);                                  /* 6) */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
      Ktot[i] = Ktot[i] + 2.0 * Ktmp[i];                          /* 7) */
      Ptmp[i] = psi[i] + dt * Ktmp[i];                            /* 8) */
    }
    evalF(&g, Ptmp, Ktmp, D, L);                                  /* 9) */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) psi[i] = psi[i] + sixth * (Ktot[i] + Ktmp[i]);  /* 10) */
  }
  free(Ktot); free(Ptmp); free(Ktmp); free(D); free(L);
  return 0;
}

/* Neumaier's compensated sum. */
typedef struct { double sum, c; } nsum;
static void nadd(nsum *acc, double x) {
  double t = acc->sum + x;
  if (fabs(acc->sum) >= fabs(x)) acc->c += (acc->sum - t) + x;
  else acc->c += (x - t) + acc->sum;
  acc->sum = t;
}

int oracle_mass(int d, const int64_t *n, double h, const double *psi, double *out) {
  int64_t total = 1;
  if (d < 1 || d > 3) return -1;
  for (int k = 0; k < d; ++k) total *= n[k];
  nsum acc = {0.0, 0.0};
  for (int64_t p = 0; p < total; ++p) {
    const double re = psi[2 * p], im = psi[2 * p + 1];
    nadd(&acc, re * re + im * im);
  }
  *out = pow(h, d) * (acc.sum + acc.c);
  return 0;
}

int oracle_energy(int d, const int64_t *n, double h, double a, double s, const double *V, int bc, int order,
                  const double *psi, double *out) {
  grid g;
  if (setup(&g, d, n, h, a, s, V, bc, order)) return -1;
  double *D = calloc(2 * g.total, sizeof(double)), *L = calloc(2 * g.total, sizeof(double));
  if (!D || !L) { free(D); free(L); return -2; }
  compute_D(&g, psi, D);
  compute_L(&g, psi, D, L);
  nsum acc = {0.0, 0.0};
  for (int64_t p = 0; p < g.total; ++p) {
    if (is_boundary(&g, p)) continue;
    const double re = psi[2 * p], im = psi[2 * p + 1];
    const double m2 = re * re + im * im;
    const double kin = -g.a * (re * L[2 * p] + im * L[2 * p + 1]);   /* -a Re(conj(Psi) Lap Psi) */
    nadd(&acc, kin + Vat(&g, p) * m2 - 0.5 * g.s * m2 * m2);
  }
  *out = pow(h, d) * (acc.sum + acc.c);
  free(D); free(L);
  return 0;
}

/* Linear stability bound for RK4 (Sec. 3.4): RK4 is stable on the imaginary
 * axis up to |z| = 2 sqrt(2); the spectral radius of a*Lap is a*rho_L with
 * rho_L = 4d/h^2 (CD) and 16d/(3h^2) (2SHOC), which gives Eqs. stblincd and
 * stblin2shoc when V = s = 0.  The potential and nonlinear terms add vmax and
 * |s| rho_max to the radius.  No safety factor is applied here. */
double oracle_stability_bound(int d, double h, double a, int order, double vmax, double s_rho_max) {
  double rho_L = (order == 4) ? 16.0 * d / (3.0 * h * h) : 4.0 * d / (h * h);
  return 2.0 * sqrt(2.0) / (a * rho_L + fabs(vmax) + fabs(s_rho_max));
}
