/*
 * Plain FP64 CPU oracle of the double-distribution thermal lattice Boltzmann
 * scheme of Hu, Zhang & Geng (arXiv 1608.06345).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline / reference arm may build, load or
 * call it; the product library never does, and the two share no code.
 *
 * Equation numbers follow the sequential numbering of the paper's revtex
 * source: Eq. (3) gamma(delta); Eq. (13a,b) the discrete reduced BGK
 * equations for g and h; Eq. (14a-c) the discrete moments; Eq. (15a,b) the
 * split of the energy; Eq. (16)/(17) the first-order time discretisation;
 * Eq. (18) the fourth-order Hermite equilibrium; Tables I and II the D2Q37 and
 * D3Q107 velocity sets; Sec. V the shock-tube set-up and the time mapping
 * t = step / (X r).
 *
 * Readings taken where the paper is garbled or silent (all listed in the
 * design notes):
 *  - Eq. (18): the printed a(k).H(k) terms for k = 2, 3, 4 are garbled (they
 *    fail even the mass moment).  The oracle uses the contraction of the
 *    Hermite coefficients of the Maxwellian with the Hermite polynomials,
 *    written out below as P2, P3, P4.
 *  - Tables I/II print weights to 9-10 digits, which leaves sum(w) - 1 at
 *    1e-8.  The oracle refines (r, w) by Newton's method on the even-moment
 *    isotropy conditions of degree 0..8, starting from the printed values.
 *  - Streaming is exact lattice streaming, x -> x + c_i per step, with the
 *    integer c_i of Tables I/II (the time mapping of Sec. V fixes
 *    dt = dx / r); the collision is the explicit BGK relaxation of
 *    Eq. (16)/(17) with 1/tau in units of dt.
 *  - "Open" ends (Sec. V) are zero-gradient: a pull from outside [0, n-1]
 *    reads the edge cell.
 *  - tau_f (for g) and tau_g (for h) may differ; the paper uses one tau.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Rounding variants.  ORA_VARIANT changes how the arithmetic below is
 * rounded, never what it computes.  The tests build the variants as second
 * checkers: how far a variant's result lies from the oracle's measures how
 * far two correct FP64 evaluations of the same scheme drift apart on a given
 * flow.  The bits of ORA_VARIANT:
 *   0  (default build) the oracle;
 *   1  every sum over the velocities runs from the last velocity to the
 *      first, and the terms of the equilibrium are added from the highest
 *      order down;
 *   2  every product-plus-sum a*b + c of the moments, the equilibrium's
 *      scalar products and the relaxation is rounded once (C99 fma);
 *   4  the relaxation q - (q - Q_eq)/tau is evaluated as
 *      (1 - 1/tau) q + (1/tau) Q_eq;
 *   8  the populations are held as deviations from the equilibrium of a
 *      reference state (rho_r, u = 0, T_r) set by ora_set_reference:
 *      dg_i = g_i - G_i, dh_i = h_i - (delta/2) T_r G_i with
 *      G_i = F_i(rho_r, 0, T_r).  The pull moves deviations, the moments add
 *      the sums of the deviations to the reference totals (rho_r for the
 *      mass, rho_r (D + delta) T_r / 2 for the energy: Eq. (14)/(15) of the
 *      reference equilibrium), and the relaxation updates the deviations
 *      towards F_i - G_i.  An exact change of variables;
 *  16  the arithmetic and the stored populations are FP32 (type real; the
 *      build adds -fsingle-precision-constant so that literals stay FP32);
 *      the velocity table is still solved in FP64 and rounded, and the
 *      grid totals of ora_conserved are still summed in FP64;
 *  32  the equilibrium is evaluated as a polynomial in s (Horner), its
 *      coefficients collected from the same Hermite terms:
 *        F_i / (w_i rho) = a0 + a1 s + a2 s^2 + s^3/6 + s^4/24,
 *        a0 = 1 - u2/2 + t (x2 - D)/2 + u2^2/8 + t (D + 2 - x2) u2/4
 *             + t^2 [x2^2 - 2 (D + 2) x2 + D (D + 2)]/8,
 *        a1 = 1 - u2/2 + t (x2 - D - 2)/2,
 *        a2 = 1/2 - u2/4 + t (x2 - D - 4)/4.
 * The default build (0) evaluates every expression exactly as written, in
 * FP64. */
#ifndef ORA_VARIANT
#define ORA_VARIANT 0
#endif
#define ORA_REV ((ORA_VARIANT) & 1)
#define ORA_FMA ((ORA_VARIANT) & 2)
#define ORA_RELAX2 ((ORA_VARIANT) & 4)
#define ORA_DEV ((ORA_VARIANT) & 8)
#define ORA_F32 ((ORA_VARIANT) & 16)
#define ORA_HORNER ((ORA_VARIANT) & 32)
#if ORA_F32
typedef float real;
#define FMA_ fmaf
#else
typedef double real;
#define FMA_ fma
#endif
#if ORA_FMA
#define MADD(a, b, c) FMA_((a), (b), (c))
#else
#define MADD(a, b, c) ((a) * (b) + (c))
#endif
/* k-th velocity of a sum over Q velocities */
#define VEL(k, Q) (ORA_REV ? (Q) - 1 - (k) : (k))

#define ORA_D2Q37 0
#define ORA_D3Q107 1
#define ORA_PERIODIC 0
#define ORA_ZERO_GRADIENT 1

/* ------------------------------------------------------------------------ */
/* Lattice: Tables I and II.                                                */
/* ------------------------------------------------------------------------ */

/* Group representatives (sorted absolute integer components) and the weights
 * as printed in Table I (D2Q37) and Table II (D3Q107), plus the printed
 * scaling factor r = 1.19697977. */
static const int d2_groups[8][2] = {
    {0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1}, {3, 0}, {3, 1}, {3, 3}};
static const double d2_printed_w[8] = {
    2.03916918e-1, 1.27544846e-1, 4.37537182e-2, 8.13659044e-3,
    9.40079914e-3, 6.95051049e-4, 3.04298494e-5, 2.81093762e-5};
static const int d3_groups[10][3] = {
    {0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {1, 1, 1}, {2, 0, 0},
    {2, 1, 1}, {2, 2, 0}, {2, 2, 2}, {3, 0, 0}, {3, 1, 1}};
static const double d3_printed_w[10] = {
    1.603003550e-1, 2.390868500e-2, 4.169870315e-2, 5.166346780e-3,
    1.227117147e-2, 2.676524495e-3, 9.685223338e-4, 2.170763000e-5,
    2.453010230e-4, 1.417071270e-4};
static const double printed_r = 1.19697977;

/* Even-moment isotropy conditions used to refine (r, w): the exponents of
 * x, y (, z).  One condition per distinct monomial class up to degree 8. */
static const int d2_mono[9][3] = {
    {0, 0, 0}, {2, 0, 0}, {4, 0, 0}, {2, 2, 0}, {6, 0, 0},
    {4, 2, 0}, {8, 0, 0}, {6, 2, 0}, {4, 4, 0}};
static const int d3_mono[11][3] = {
    {0, 0, 0}, {2, 0, 0}, {4, 0, 0}, {2, 2, 0}, {6, 0, 0}, {4, 2, 0},
    {2, 2, 2}, {8, 0, 0}, {6, 2, 0}, {4, 4, 0}, {4, 2, 2}};

typedef struct {
  int D, Q, G;      /* dimension, velocities, groups */
  int c[107][3];    /* integer velocities c_i (z = 0 in 2D) */
  int group[107];   /* group index of velocity i */
  double w[107];    /* refined weight of velocity i */
  double wg[10];    /* refined weight per group */
  double r;         /* refined scaling factor; xi_i = r c_i */
} ora_lattice_t;

static int iabs_(int a) { return a < 0 ? -a : a; }

/* Which group a velocity belongs to: its sorted absolute components must
 * equal a representative; -1 if none. */
static int group_of(int D, const int* v) {
  int a[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) a[k] = iabs_(v[k]);
  /* sort descending */
  for (int p = 0; p < D; ++p)
    for (int q = p + 1; q < D; ++q)
      if (a[q] > a[p]) { int t = a[p]; a[p] = a[q]; a[q] = t; }
  if (D == 2) {
    for (int g = 0; g < 8; ++g)
      if (a[0] == d2_groups[g][0] && a[1] == d2_groups[g][1]) return g;
  } else {
    for (int g = 0; g < 10; ++g)
      if (a[0] == d3_groups[g][0] && a[1] == d3_groups[g][1] &&
          a[2] == d3_groups[g][2])
        return g;
  }
  return -1;
}

static double ipow_(double x, int n) {
  double p = 1.0;
  for (int k = 0; k < n; ++k) p *= x;
  return p;
}

/* (n-1)!! : the n-th moment of the unit Gaussian (n even), 0 for n odd. */
static double gauss_moment(int n) {
  if (n % 2) return 0.0;
  double m = 1.0;
  for (int k = n - 1; k > 1; k -= 2) m *= k;
  return m;
}

/* Solve A x = b (n x n, row-major) by Gaussian elimination with partial
 * pivoting.  A and b are overwritten.  Returns 0 on success. */
static int solve_dense(int n, double* A, double* b, double* x) {
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int row = col + 1; row < n; ++row)
      if (fabs(A[row * n + col]) > fabs(A[piv * n + col])) piv = row;
    if (A[piv * n + col] == 0.0) return -1;
    if (piv != col) {
      for (int k = 0; k < n; ++k) {
        double t = A[col * n + k]; A[col * n + k] = A[piv * n + k]; A[piv * n + k] = t;
      }
      double t = b[col]; b[col] = b[piv]; b[piv] = t;
    }
    for (int row = col + 1; row < n; ++row) {
      double f = A[row * n + col] / A[col * n + col];
      for (int k = col; k < n; ++k) A[row * n + k] -= f * A[col * n + k];
      b[row] -= f * b[col];
    }
  }
  for (int row = n - 1; row >= 0; --row) {
    double s = b[row];
    for (int k = row + 1; k < n; ++k) s -= A[row * n + k] * x[k];
    x[row] = s / A[row * n + row];
  }
  return 0;
}

/* Double-double numbers (hi + lo, |lo| <= ulp(hi)/2) for the residuals of
 * the refinement: the error-free transformations of Knuth (two_sum) and of
 * Dekker with a fused multiply-add (two_prod). */
typedef struct { double hi, lo; } dd_t;

static dd_t two_sum(double a, double b) {
  dd_t r;
  r.hi = a + b;
  double bb = r.hi - a;
  r.lo = (a - (r.hi - bb)) + (b - bb);
  return r;
}

static dd_t two_prod(double a, double b) {
  dd_t r;
  r.hi = a * b;
  r.lo = fma(a, b, -r.hi);
  return r;
}

static dd_t dd_add(dd_t a, dd_t b) {
  dd_t s = two_sum(a.hi, b.hi);
  return two_sum(s.hi, s.lo + a.lo + b.lo);
}

static dd_t dd_mul(dd_t a, dd_t b) {
  dd_t p = two_prod(a.hi, b.hi);
  return two_sum(p.hi, p.lo + a.hi * b.lo + a.lo * b.hi);
}

/* Residual of one isotropy condition, r^deg sum_g w_g M_g - target, in
 * double-double. */
static double isotropy_residual(int G, const double* w, double r, int deg, const double* M,
                                double target) {
  dd_t sw = {0.0, 0.0};
  for (int g = 0; g < G; ++g) sw = dd_add(sw, two_prod(w[g], M[g]));
  dd_t rp = {1.0, 0.0};
  for (int k = 0; k < deg; ++k) rp = dd_mul(rp, (dd_t){r, 0.0});
  dd_t v = dd_add(dd_mul(rp, sw), (dd_t){-target, 0.0});
  return v.hi + v.lo;
}

/* Build the velocity set of Table I / II and refine (r, w).
 *
 * Velocities: every integer vector in {-3..3}^D whose sorted absolute values
 * equal a group representative (the "Perm" rows of the tables), ordered by
 * group, then lexicographically.
 *
 * Refinement: the unknowns are the G group weights and r; the conditions are
 * sum_i w_i (r c_i)^alpha = E[xi^alpha] of the unit Gaussian for the G+1
 * monomial classes listed above.  Newton's method with the exact Jacobian,
 * from the printed values; then three more Newton corrections whose
 * residuals are evaluated in double-double arithmetic.  The system is
 * ill-conditioned in the smallest weights, so residuals in double leave
 * the weights uncertain by up to 1e-13 relative (about a thousand ulps);
 * with accurate residuals each correction removes the remaining error, and
 * the result is the solution of the conditions rounded to double. */
static int build_lattice(int lattice, ora_lattice_t* L) {
  memset(L, 0, sizeof(*L));
  if (lattice == ORA_D2Q37) { L->D = 2; L->G = 8; }
  else if (lattice == ORA_D3Q107) { L->D = 3; L->G = 10; }
  else return -1;
  const int D = L->D, G = L->G;
  int q = 0;
  for (int g = 0; g < G; ++g) {
    int v[3];
    int zr = (D == 3) ? 3 : 0;
    for (v[0] = -3; v[0] <= 3; ++v[0])
      for (v[1] = -3; v[1] <= 3; ++v[1])
        for (v[2] = -zr; v[2] <= zr; ++v[2]) {
          if (group_of(D, v) != g) continue;
          for (int k = 0; k < 3; ++k) L->c[q][k] = (k < D) ? v[k] : 0;
          L->group[q] = g;
          ++q;
        }
  }
  L->Q = q;
  if ((D == 2 && q != 37) || (D == 3 && q != 107)) return -2;

  /* M[k][g] = sum over the velocities of group g of c^alpha_k (integer). */
  const int (*mono)[3] = (D == 2) ? d2_mono : d3_mono;
  const int K = G + 1;
  double M[11][10];
  int deg[11];
  double target[11];
  for (int k = 0; k < K; ++k) {
    deg[k] = mono[k][0] + mono[k][1] + mono[k][2];
    target[k] = gauss_moment(mono[k][0]) * gauss_moment(mono[k][1]) *
                gauss_moment(mono[k][2]);
    for (int g = 0; g < G; ++g) M[k][g] = 0.0;
    for (int i = 0; i < q; ++i) {
      double m = ipow_(L->c[i][0], mono[k][0]) * ipow_(L->c[i][1], mono[k][1]) *
                 ipow_(L->c[i][2], mono[k][2]);
      M[k][L->group[i]] += m;
    }
  }
  double x[11];
  for (int g = 0; g < G; ++g) x[g] = (D == 2) ? d2_printed_w[g] : d3_printed_w[g];
  x[G] = printed_r;
  for (int it = 0; it < 50; ++it) {
    double A[121], b[11], dx[11];
    double r = x[G];
    for (int k = 0; k < K; ++k) {
      double sw = 0.0;
      for (int g = 0; g < G; ++g) sw += x[g] * M[k][g];
      /* residual R_k = r^deg sum_g w_g M_kg - target_k */
      b[k] = -(ipow_(r, deg[k]) * sw - target[k]);
      for (int g = 0; g < G; ++g) A[k * K + g] = ipow_(r, deg[k]) * M[k][g];
      A[k * K + G] = (deg[k] > 0) ? deg[k] * ipow_(r, deg[k] - 1) * sw : 0.0;
    }
    if (solve_dense(K, A, b, dx)) return -3;
    double step = 0.0;
    for (int k = 0; k < K; ++k) {
      x[k] += dx[k];
      step = fmax(step, fabs(dx[k]) / fabs(x[k]));
    }
    if (step < 1e-16) break;
  }
  for (int it = 0; it < 3; ++it) {
    double A[121], b[11], dx[11];
    double r = x[G];
    for (int k = 0; k < K; ++k) {
      double sw = 0.0;
      for (int g = 0; g < G; ++g) sw += x[g] * M[k][g];
      b[k] = -isotropy_residual(G, x, r, deg[k], M[k], target[k]);
      for (int g = 0; g < G; ++g) A[k * K + g] = ipow_(r, deg[k]) * M[k][g];
      A[k * K + G] = (deg[k] > 0) ? deg[k] * ipow_(r, deg[k] - 1) * sw : 0.0;
    }
    if (solve_dense(K, A, b, dx)) return -3;
    for (int k = 0; k < K; ++k) x[k] += dx[k];
  }
  for (int g = 0; g < G; ++g) L->wg[g] = x[g];
  L->r = x[G];
  for (int i = 0; i < q; ++i) L->w[i] = L->wg[L->group[i]];
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Equilibrium, Eq. (18), with the derived Hermite contractions.            */
/* ------------------------------------------------------------------------ */

/* F_i = w_i rho sum_{k=0..4} a(k).H(k)(xi_i) / k!, where, with s = xi.u,
 * u2 = |u|^2, x2 = |xi|^2 and t = theta - 1 (theta = T):
 *   a0.H0 = 1
 *   a1.H1 = s
 *   a2.H2 = s^2 - u2 + t (x2 - D)
 *   a3.H3 = s [s^2 - 3 u2 + 3 t (x2 - D - 2)]
 *   a4.H4 = s^4 - 6 s^2 u2 + 3 u2^2
 *           + 6 t [s^2 (x2 - D - 4) + (D + 2 - x2) u2]
 *           + 3 t^2 [x2^2 - 2 (D + 2) x2 + D (D + 2)]
 * These are the contractions of the Maxwellian's Hermite coefficients
 * a(2) = uu + t I, a(3) = uuu + t sym(uI), a(4) = uuuu + t sym(uuI)
 * + t^2 sym(II) with the tensor Hermite polynomials. */
static void equilibrium(const ora_lattice_t* L, real rho, const real* u,
                        real T, real* F) {
  const int D = L->D;
  real u2 = 0.0;
  for (int a = 0; a < D; ++a) u2 += u[a] * u[a];
  const real t = T - 1.0;
  for (int i = 0; i < L->Q; ++i) {
    real s = 0.0, x2 = 0.0;
    for (int a = 0; a < D; ++a) {
      real xi = (real)L->r * L->c[i][a];
      s = MADD(xi, u[a], s);
      x2 = MADD(xi, xi, x2);
    }
    real h0 = 1.0;
    real h1 = s;
    real h2 = s * s - u2 + t * (x2 - D);
    real h3 = s * (s * s - 3.0 * u2 + 3.0 * t * (x2 - D - 2.0));
    real h4 = s * s * s * s - 6.0 * s * s * u2 + 3.0 * u2 * u2 +
              6.0 * t * (s * s * (x2 - D - 4.0) + (D + 2.0 - x2) * u2) +
              3.0 * t * t * (x2 * x2 - 2.0 * (D + 2.0) * x2 + D * (D + 2.0));
#if ORA_HORNER
    const real a0 = 1.0 - u2 / 2.0 + t * (x2 - D) / 2.0 + u2 * u2 / 8.0 + t * (D + 2.0 - x2) * u2 / 4.0 +
                    t * t * (x2 * x2 - 2.0 * (D + 2.0) * x2 + D * (D + 2.0)) / 8.0;
    const real a1 = 1.0 - u2 / 2.0 + t * (x2 - D - 2.0) / 2.0;
    const real a2 = 0.5 - u2 / 4.0 + t * (x2 - D - 4.0) / 4.0;
    (void)h0; (void)h1; (void)h2; (void)h3; (void)h4;
    F[i] = (real)L->w[i] * rho * ((((s / 24.0 + 1.0 / 6.0) * s + a2) * s + a1) * s + a0);
#elif ORA_REV
    F[i] = (real)L->w[i] * rho * (h4 / 24.0 + h3 / 6.0 + h2 / 2.0 + h1 + h0);
#else
    F[i] = (real)L->w[i] * rho * (h0 + h1 + h2 / 2.0 + h3 / 6.0 + h4 / 24.0);
#endif
  }
}

/* Moments of one cell, Eq. (14a-c) and Eq. (15a,b):
 *   rho = sum g_i, rho u = sum xi_i g_i, rho E = sum xi_i^2 g_i / 2 + sum h_i,
 *   E = u^2/2 + (D + delta)/2 T  =>  T = 2 (E - u^2/2) / (D + delta).
 * m0, e0 are added to the mass and energy sums: 0 in the oracle, whose
 * populations are stored whole; the reference totals in variant 8. */
static void cell_moments(const ora_lattice_t* L, real delta, real m0, real e0,
                         const real* g, const real* h, real* rho, real* u, real* T) {
  const int D = L->D;
  real r0 = m0, j[3] = {0.0, 0.0, 0.0}, e = e0;
  for (int k = 0; k < L->Q; ++k) {
    const int i = VEL(k, L->Q);
    real x2 = 0.0;
    for (int a = 0; a < D; ++a) {
      real xi = (real)L->r * L->c[i][a];
      j[a] = MADD(xi, g[i], j[a]);
      x2 = MADD(xi, xi, x2);
    }
    r0 += g[i];
    e += MADD(0.5 * x2, g[i], h[i]);
  }
  real u2 = 0.0;
  for (int a = 0; a < D; ++a) {
    u[a] = j[a] / r0;
    u2 += u[a] * u[a];
  }
  *rho = r0;
  *T = 2.0 * (e / r0 - 0.5 * u2) / (D + delta);
}

/* ------------------------------------------------------------------------ */
/* Solver state.                                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
  ora_lattice_t L;
  double delta, tau_f, tau_g;
  int n[3];        /* nx, ny, nz (nz = 1 in 2D) */
  int bc[3];       /* per axis: periodic or zero-gradient */
  long N;          /* cells */
  real *g, *h;     /* populations, g[i * N + cell] */
  real *g2, *h2;   /* second buffer */
  /* variant 8 only: the reference equilibrium G_i, (delta/2) T_r G_i and its
   * mass and energy totals; zero in the oracle */
  real ref_g[107], ref_h[107], ref_m, ref_e;
} ora_state;

int ora_set_reference(ora_state* s, double rho_r, double T_r);

/* delta from gamma, Eq. (3): gamma = (delta + D + 2) / (delta + D). */
double ora_delta_from_gamma(int D, double gamma) {
  return 2.0 / (gamma - 1.0) - D;
}

int ora_lattice_info(int lattice, int* Q, int* c, double* w, double* r) {
  ora_lattice_t L;
  int rc = build_lattice(lattice, &L);
  if (rc) return rc;
  if (Q) *Q = L.Q;
  for (int i = 0; i < L.Q; ++i) {
    if (c)
      for (int a = 0; a < L.D; ++a) c[i * L.D + a] = L.c[i][a];
    if (w) w[i] = L.w[i];
  }
  if (r) *r = L.r;
  return 0;
}

/* Equilibrium of one state (rho, u[D], T) into F[Q]; for tests. */
int ora_feq(int lattice, double rho, const double* u, double T, double* F) {
  ora_lattice_t L;
  int rc = build_lattice(lattice, &L);
  if (rc) return rc;
  real ur[3] = {0.0, 0.0, 0.0}, Fr[107];
  for (int a = 0; a < L.D; ++a) ur[a] = (real)u[a];
  equilibrium(&L, (real)rho, ur, (real)T, Fr);
  for (int i = 0; i < L.Q; ++i) F[i] = Fr[i];
  return 0;
}

void ora_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int ora_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void ora_free(ora_state* s) {
  if (!s) return;
  free(s->g); free(s->h); free(s->g2); free(s->h2);
  free(s);
}

ora_state* ora_new(int lattice, double gamma, double tau_f, double tau_g,
                   int nx, int ny, int nz, int bcx, int bcy, int bcz) {
  ora_state* s = (ora_state*)calloc(1, sizeof(ora_state));
  if (!s) return NULL;
  if (build_lattice(lattice, &s->L)) { free(s); return NULL; }
  if (s->L.D == 2 && nz != 1) { free(s); return NULL; }
  if (nx < 1 || ny < 1 || nz < 1) { free(s); return NULL; }
  s->delta = ora_delta_from_gamma(s->L.D, gamma);
  s->tau_f = tau_f;
  s->tau_g = tau_g;
  s->n[0] = nx; s->n[1] = ny; s->n[2] = nz;
  s->bc[0] = bcx; s->bc[1] = bcy; s->bc[2] = bcz;
  s->N = (long)nx * ny * nz;
#if ORA_DEV
  ora_set_reference(s, 1.0, 1.0);
#endif
  size_t bytes = sizeof(real) * (size_t)s->L.Q * (size_t)s->N;
  s->g = (real*)malloc(bytes);
  s->h = (real*)malloc(bytes);
  s->g2 = (real*)malloc(bytes);
  s->h2 = (real*)malloc(bytes);
  if (!s->g || !s->h || !s->g2 || !s->h2) { ora_free(s); return NULL; }
  return s;
}

double ora_delta(const ora_state* s) { return s->delta; }

/* Initial state: g_i = F_i(rho, u, T), h_i = (delta/2) T F_i (Eq. (13b)'s
 * equilibrium), cell by cell.  u is component-major: u[a * N + cell]. */
void ora_init(ora_state* s, const double* rho, const double* u, const double* T) {
  const long N = s->N;
  const int Q = s->L.Q, D = s->L.D;
  const real hd = (real)(0.5 * s->delta);
#pragma omp parallel for schedule(static)
  for (long cell = 0; cell < N; ++cell) {
    real F[107], uc[3];
    const real Tc = (real)T[cell];
    for (int a = 0; a < D; ++a) uc[a] = (real)u[a * N + cell];
    equilibrium(&s->L, (real)rho[cell], uc, Tc, F);
    for (int i = 0; i < Q; ++i) {
#if ORA_DEV
      s->g[i * N + cell] = F[i] - s->ref_g[i];
      s->h[i * N + cell] = hd * Tc * F[i] - s->ref_h[i];
#else
      s->g[i * N + cell] = F[i];
      s->h[i * N + cell] = hd * Tc * F[i];
#endif
    }
  }
}

/* Source index along one axis for a pull from position p - c. */
static int pull_index(int p, int c, int n, int bc) {
  int q = p - c;
  if (bc == ORA_PERIODIC) {
    q %= n;
    if (q < 0) q += n;
  } else {
    if (q < 0) q = 0;
    if (q > n - 1) q = n - 1;
  }
  return q;
}

/* One time step for every cell:
 *   pull   g~_i(x) = g*_i(x - c_i),  h~_i(x) = h*_i(x - c_i)
 *   moments of (g~, h~)                                  Eq. (14), (15)
 *   F_i = equilibrium(rho, u, T),  Fh_i = (delta/2) T F_i  Eq. (18), (13b)
 *   g*_i = g~_i - (1/tau_f)(g~_i - F_i)                   Eq. (16)
 *   h*_i = h~_i - (1/tau_g)(h~_i - Fh_i)                  Eq. (17)
 * then the buffers swap. */
static void step_once(ora_state* s) {
  const long N = s->N;
  const int Q = s->L.Q, D = s->L.D;
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  const real wf = (real)(1.0 / s->tau_f), wg = (real)(1.0 / s->tau_g);
  const real hd = (real)(0.5 * s->delta);
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y) {
      real gt[107], ht[107], F[107], u[3], rho, T;
      for (int x = 0; x < nx; ++x) {
        long cell = x + (long)nx * (y + (long)ny * z);
        for (int i = 0; i < Q; ++i) {
          int sx = pull_index(x, s->L.c[i][0], nx, s->bc[0]);
          int sy = pull_index(y, s->L.c[i][1], ny, s->bc[1]);
          int sz = pull_index(z, s->L.c[i][2], nz, s->bc[2]);
          long src = sx + (long)nx * (sy + (long)ny * sz);
          gt[i] = s->g[i * N + src];
          ht[i] = s->h[i * N + src];
        }
        cell_moments(&s->L, (real)s->delta, s->ref_m, s->ref_e, gt, ht, &rho, u, &T);
        equilibrium(&s->L, rho, u, T, F);
        for (int i = 0; i < Q; ++i) {
          real Fh = hd * T * F[i];
#if ORA_DEV
          Fh -= s->ref_h[i];
          F[i] -= s->ref_g[i];
#endif
#if ORA_RELAX2
          s->g2[i * N + cell] = MADD(1.0 - wf, gt[i], wf * F[i]);
          s->h2[i * N + cell] = MADD(1.0 - wg, ht[i], wg * Fh);
#else
          s->g2[i * N + cell] = MADD(-wf, gt[i] - F[i], gt[i]);
          s->h2[i * N + cell] = MADD(-wg, ht[i] - Fh, ht[i]);
#endif
        }
      }
    }
  (void)D;
  real* t;
  t = s->g; s->g = s->g2; s->g2 = t;
  t = s->h; s->h = s->h2; s->h2 = t;
}

void ora_step(ora_state* s, long nsteps) {
  for (long k = 0; k < nsteps; ++k) step_once(s);
}

/* ------------------------------------------------------------------------ */
/* Finite-difference variant of Sec. III: Eq. (16)/(17) with the convection */
/* term discretised by the third-order upwind scheme along each axis.       */
/* ------------------------------------------------------------------------ */

/* Third-order upwind approximation of dq/dx at p along one axis, for a
 * velocity component of sign `sgn` (Sec. III; the printed g_j is read as
 * g_i):
 *   sgn > 0:  [q(p-2) - 6 q(p-1) + 3 q(p) + 2 q(p+1)] / 6
 *   sgn < 0:  [-q(p+2) + 6 q(p+1) - 3 q(p) - 2 q(p-1)] / 6
 * Neighbours outside the grid follow the axis' boundary rule (periodic wrap
 * or the edge cell).  `at(k)` reads q at axis position k. */
static real upwind3(int p, int sgn, int n, int bc, const real* plane, long stride, long base) {
#define Q_AT(k) plane[base + (long)pull_index((p), -(k), (n), (bc)) * stride]
  real d;
  if (sgn > 0)
    d = (Q_AT(-2) - 6.0 * Q_AT(-1) + 3.0 * Q_AT(0) + 2.0 * Q_AT(1)) / 6.0;
  else
    d = (-Q_AT(2) + 6.0 * Q_AT(1) - 3.0 * Q_AT(0) - 2.0 * Q_AT(-1)) / 6.0;
#undef Q_AT
  return d;
}

/* One forward-Euler step of Eq. (16)/(17) with lambda = dt/dx:
 *   g_i <- g_i - lambda sum_a xi_ia D_a(g_i) - (1/tau_f)(g_i - F_i)
 *   h_i <- h_i - lambda sum_a xi_ia D_a(h_i) - (1/tau_g)(h_i - (delta/2) T F_i)
 * with D_a the third-order upwind difference along axis a for the sign of
 * xi_ia, and F, T from the cell's own moments at the old time level. */
static void step_fd_once(ora_state* s, double lambda) {
  const long N = s->N;
  const int Q = s->L.Q, D = s->L.D;
  const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
  const long stride[3] = {1, nx, (long)nx * ny};
  const real wf = (real)(1.0 / s->tau_f), wg = (real)(1.0 / s->tau_g);
  const real hd = (real)(0.5 * s->delta), lam = (real)lambda;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y) {
      real gc[107], hc[107], F[107], u[3], rho, T;
      for (int x = 0; x < nx; ++x) {
        const long cell = x + (long)nx * (y + (long)ny * z);
        const int pos[3] = {x, y, z};
        const int nn[3] = {nx, ny, nz};
        for (int i = 0; i < Q; ++i) {
          gc[i] = s->g[i * N + cell];
          hc[i] = s->h[i * N + cell];
        }
        cell_moments(&s->L, (real)s->delta, s->ref_m, s->ref_e, gc, hc, &rho, u, &T);
        equilibrium(&s->L, rho, u, T, F);
        for (int i = 0; i < Q; ++i) {
          real cg = 0.0, ch = 0.0;
          for (int a = 0; a < D; ++a) {
            const int c = s->L.c[i][a];
            if (c == 0) continue;
            const real xi = (real)s->L.r * c;
            const long base = cell - (long)pos[a] * stride[a];
            cg += xi * upwind3(pos[a], c, nn[a], s->bc[a], s->g + i * N, stride[a], base);
            ch += xi * upwind3(pos[a], c, nn[a], s->bc[a], s->h + i * N, stride[a], base);
          }
#if ORA_DEV
          const real Fh = hd * T * F[i] - s->ref_h[i];
          F[i] -= s->ref_g[i];
#else
          const real Fh = hd * T * F[i];
#endif
          s->g2[i * N + cell] = gc[i] - lam * cg - wf * (gc[i] - F[i]);
          s->h2[i * N + cell] = hc[i] - lam * ch - wg * (hc[i] - Fh);
        }
      }
    }
  real* t;
  t = s->g; s->g = s->g2; s->g2 = t;
  t = s->h; s->h = s->h2; s->h2 = t;
}

void ora_step_fd(ora_state* s, long nsteps, double lambda) {
  for (long k = 0; k < nsteps; ++k) step_fd_once(s, lambda);
}

/* rho, u (component-major), T of the stored state, per cell. */
void ora_moments(const ora_state* s, double* rho, double* u, double* T) {
  const long N = s->N;
  const int Q = s->L.Q, D = s->L.D;
#pragma omp parallel for schedule(static)
  for (long cell = 0; cell < N; ++cell) {
    real g[107], h[107], uc[3], rc, Tc;
    for (int i = 0; i < Q; ++i) {
      g[i] = s->g[i * N + cell];
      h[i] = s->h[i * N + cell];
    }
    cell_moments(&s->L, (real)s->delta, s->ref_m, s->ref_e, g, h, &rc, uc, &Tc);
    rho[cell] = rc;
    T[cell] = Tc;
    for (int a = 0; a < D; ++a) u[a * N + cell] = uc[a];
  }
}

/* Neumaier's compensated summation (Neumaier 1974): the running sum s and
 * the accumulated rounding error c of its additions; the total is s + c. */
typedef struct { double s, c; } ksum_t;

static void ksum_add(ksum_t* k, double v) {
  const double t = k->s + v;
  if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
  else k->c += (v - t) + k->s;
  k->s = t;
}

/* Grid totals of the stored state: out = [mass, momentum[D], energy] with
 * mass = sum g, momentum = sum xi g, energy = sum (xi^2/2 g + h), Eq. (14).
 * Summed in cell order with compensated sums: a plain running sum over the
 * Q N terms of a grid drifts by up to ~1e-12 relative (measured on a 1024-cell
 * D3Q107 tube), more than the round-off the conservation pins resolve. */
void ora_conserved(const ora_state* s, double* out) {
  const long N = s->N;
  const int Q = s->L.Q, D = s->L.D;
  ksum_t m = {0.0, 0.0}, j[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}}, e = {0.0, 0.0};
  for (long cell = 0; cell < N; ++cell)
    for (int i = 0; i < Q; ++i) {
      double gi = s->g[i * N + cell], hi = s->h[i * N + cell];
#if ORA_DEV
      gi += s->ref_g[i];
      hi += s->ref_h[i];
#endif
      double x2 = 0.0;
      for (int a = 0; a < D; ++a) {
        double xi = s->L.r * s->L.c[i][a];
        ksum_add(&j[a], xi * gi);
        x2 += xi * xi;
      }
      ksum_add(&m, gi);
      ksum_add(&e, 0.5 * x2 * gi + hi);
    }
  out[0] = m.s + m.c;
  for (int a = 0; a < D; ++a) out[1 + a] = j[a].s + j[a].c;
  out[1 + D] = e.s + e.c;
}

/* Direct access to the populations, [i * N + cell], in the oracle's own
 * velocity order (ora_lattice_info). */
void ora_get_pops(const ora_state* s, double* g, double* h) {
  const long n = (long)s->L.Q * s->N;
  for (long k = 0; k < n; ++k) {
    g[k] = s->g[k];
    h[k] = s->h[k];
  }
#if ORA_DEV
  for (int i = 0; i < s->L.Q; ++i)
    for (long cell = 0; cell < s->N; ++cell) {
      g[i * s->N + cell] += s->ref_g[i];
      h[i * s->N + cell] += s->ref_h[i];
    }
#endif
}

void ora_set_pops(ora_state* s, const double* g, const double* h) {
  const long n = (long)s->L.Q * s->N;
  for (long k = 0; k < n; ++k) {
    s->g[k] = (real)g[k];
    s->h[k] = (real)h[k];
  }
#if ORA_DEV
  for (int i = 0; i < s->L.Q; ++i)
    for (long cell = 0; cell < s->N; ++cell) {
      s->g[i * s->N + cell] -= s->ref_g[i];
      s->h[i * s->N + cell] -= s->ref_h[i];
    }
#endif
}

/* Reference state of variant 8 (rho_r, u = 0, T_r); the default is (1, 1).
 * Call before ora_init.  Returns -1 in builds without variant 8, whose
 * populations are stored whole. */
int ora_set_reference(ora_state* s, double rho_r, double T_r) {
#if ORA_DEV
  const real zero[3] = {0.0, 0.0, 0.0};
  const real hd = (real)(0.5 * s->delta);
  equilibrium(&s->L, (real)rho_r, zero, (real)T_r, s->ref_g);
  for (int i = 0; i < s->L.Q; ++i) s->ref_h[i] = hd * (real)T_r * s->ref_g[i];
  s->ref_m = (real)rho_r;
  s->ref_e = (real)(0.5 * rho_r * (s->L.D + s->delta) * T_r);
  return 0;
#else
  (void)s; (void)rho_r; (void)T_r;
  return -1;
#endif
}
