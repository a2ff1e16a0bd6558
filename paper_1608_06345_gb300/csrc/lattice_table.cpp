// Host FP64 lattice table: refined weights and scaling factor of the
// D2Q37 (Table I) and D3Q107 (Table II) Hermite quadratures.
//
// The tables print r and the weights to 9-10 digits, which leaves the mass
// moment off by 1e-8 and would make FP64 runs drift.  The table is therefore
// recomputed from its defining property: the weighted velocity moments
// sum_i w_i xi_i^alpha must equal those of the unit Gaussian for the
// even-moment classes of degree 0..8 (G+1 conditions for G weights and r).
//
// Method: for a fixed r the conditions are linear in the group weights.
// All conditions but x^8 determine w(r) by a dense solve; r is then the root
// of the remaining x^8 condition, found by the secant method from [1.19, 1.20]
// (the printed r is 1.19697977).  The conditions are ill-conditioned in the
// smallest weights: solved with residuals in double, the weights are only
// determined to about 1e-13 relative.  A final refinement therefore
// evaluates the residuals of all G+1 conditions in double-double arithmetic
// and corrects (w, r) with the Jacobian of the full system, which leaves the
// solution of the conditions rounded to double.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <vector>

#include "lattice.h"

namespace lbm {
namespace {

double gaussian_moment(int n) {  // (n-1)!! for even n
  if (n % 2) return 0.0;
  double m = 1.0;
  for (int k = n - 1; k > 1; k -= 2) m *= k;
  return m;
}

// Dense LU solve with partial pivoting; returns false if singular.
bool lu_solve(int n, double* a, double* b) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(a[i * n + k]) > std::fabs(a[p * n + k])) p = i;
    if (a[p * n + k] == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(a[k * n + j], a[p * n + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      double l = a[i * n + k] / a[k * n + k];
      a[i * n + k] = 0.0;
      for (int j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= a[i * n + j] * b[j];
    b[i] = s / a[i * n + i];
  }
  return true;
}

// Double-double values (hi + lo) for the residuals of the final refinement:
// error-free sum (Knuth) and product (Dekker, with a fused multiply-add).
struct DD {
  double hi, lo;
};

DD dd_two_sum(double a, double b) {
  const double s = a + b;
  const double bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

DD dd_two_prod(double a, double b) {
  const double p = a * b;
  return {p, std::fma(a, b, -p)};
}

DD dd_add(DD a, DD b) {
  const DD s = dd_two_sum(a.hi, b.hi);
  return dd_two_sum(s.hi, s.lo + a.lo + b.lo);
}

DD dd_mul(DD a, DD b) {
  const DD p = dd_two_prod(a.hi, b.hi);
  return dd_two_sum(p.hi, p.lo + a.hi * b.lo + a.lo * b.hi);
}

struct Problem {
  const LatticeDef* L;
  int nlin;              // conditions solved linearly (= G)
  int mono[11][3];       // exponents; mono[nlin] is the secant condition x^8
};

// sum over the members of group g of (r c)^alpha
double group_moment(const LatticeDef& L, int g, const int* alpha, double r) {
  double s = 0.0;
  for (int i = 0; i < L.Q; ++i) {
    if (L.grp[i] != g) continue;
    double m = 1.0;
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < alpha[a]; ++k) m *= r * L.c[i][a];
    s += m;
  }
  return s;
}

double target(const int* alpha) {
  return gaussian_moment(alpha[0]) * gaussian_moment(alpha[1]) * gaussian_moment(alpha[2]);
}

// Weights for a given r (linear conditions); returns the x^8 residual.
bool weights_for(const Problem& P, double r, double* w, double* resid) {
  const LatticeDef& L = *P.L;
  const int n = P.nlin;
  double a[100], b[10];
  for (int k = 0; k < n; ++k) {
    for (int g = 0; g < n; ++g) a[k * n + g] = group_moment(L, g, P.mono[k], r);
    b[k] = target(P.mono[k]);
  }
  if (!lu_solve(n, a, b)) return false;
  double s = 0.0;
  for (int g = 0; g < n; ++g) {
    w[g] = b[g];
    s += w[g] * group_moment(L, g, P.mono[n], r);
  }
  *resid = s - target(P.mono[n]);
  return true;
}

// integer moment of group g: sum over its members of c^alpha (exact)
double group_moment_int(const LatticeDef& L, int g, const int* alpha) {
  long long s = 0;
  for (int i = 0; i < L.Q; ++i) {
    if (L.grp[i] != g) continue;
    long long m = 1;
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < alpha[a]; ++k) m *= L.c[i][a];
    s += m;
  }
  return (double)s;
}

// Newton corrections of (w, r) on all G+1 conditions with residuals in
// double-double: R_k = r^d_k sum_g w_g M_kg - target_k, J = dR/d(w, r).
bool refine_dd(const Problem& P, double* w, double* r, int iters) {
  const LatticeDef& L = *P.L;
  const int G = P.nlin, K = G + 1;
  double M[11][10];
  int deg[11];
  for (int k = 0; k < K; ++k) {
    deg[k] = P.mono[k][0] + P.mono[k][1] + P.mono[k][2];
    for (int g = 0; g < G; ++g) M[k][g] = group_moment_int(L, g, P.mono[k]);
  }
  for (int it = 0; it < iters; ++it) {
    double a[121], b[11];
    for (int k = 0; k < K; ++k) {
      DD sw{0.0, 0.0};
      double swd = 0.0;
      for (int g = 0; g < G; ++g) {
        sw = dd_add(sw, dd_two_prod(w[g], M[k][g]));
        swd += w[g] * M[k][g];
      }
      DD rp{1.0, 0.0};
      double rpd = 1.0, rpd1 = 1.0;  // r^d and r^(d-1) in double for the Jacobian
      for (int q = 0; q < deg[k]; ++q) {
        rp = dd_mul(rp, DD{*r, 0.0});
        if (q + 1 < deg[k]) rpd1 *= *r;
        rpd *= *r;
      }
      const DD res = dd_add(dd_mul(rp, sw), DD{-target(P.mono[k]), 0.0});
      b[k] = -(res.hi + res.lo);
      for (int g = 0; g < G; ++g) a[k * K + g] = rpd * M[k][g];
      a[k * K + G] = deg[k] > 0 ? deg[k] * rpd1 * swd : 0.0;
    }
    if (!lu_solve(K, a, b)) return false;
    for (int g = 0; g < G; ++g) w[g] += b[g];
    *r += b[G];
  }
  return true;
}

}  // namespace

static int build_lattice_table_uncached(int lattice, LatticeTable* out) {
  Problem P{};
  if (lattice == 0) {
    static const int m[9][3] = {{0, 0, 0}, {2, 0, 0}, {4, 0, 0}, {2, 2, 0}, {6, 0, 0},
                                {4, 2, 0}, {6, 2, 0}, {4, 4, 0}, {8, 0, 0}};
    P.L = &kD2Q37;
    P.nlin = 8;
    std::memcpy(P.mono, m, sizeof(m));
  } else if (lattice == 1) {
    static const int m[11][3] = {{0, 0, 0}, {2, 0, 0}, {4, 0, 0}, {2, 2, 0}, {6, 0, 0}, {4, 2, 0},
                                 {2, 2, 2}, {6, 2, 0}, {4, 4, 0}, {4, 2, 2}, {8, 0, 0}};
    P.L = &kD3Q107;
    P.nlin = 10;
    std::memcpy(P.mono, m, sizeof(m));
  } else {
    return -1;
  }
  double w[10];
  double r0 = 1.19, r1 = 1.20, f0, f1;
  if (!weights_for(P, r0, w, &f0) || !weights_for(P, r1, w, &f1)) return -2;
  for (int it = 0; it < 100 && f1 != f0; ++it) {
    double r2 = r1 - f1 * (r1 - r0) / (f1 - f0);
    r0 = r1;
    f0 = f1;
    r1 = r2;
    if (!weights_for(P, r1, w, &f1)) return -2;
    if (std::fabs(r1 - r0) <= 1e-16 * r1) break;
  }
  if (!weights_for(P, r1, w, &f1)) return -2;
  if (!refine_dd(P, w, &r1, 3)) return -2;
  const LatticeDef& L = *P.L;
  out->D = L.D;
  out->Q = L.Q;
  out->G = L.G;
  out->r = r1;
  for (int g = 0; g < L.G; ++g) {
    out->wg[g] = w[g];
    out->x2g[g] = r1 * r1 * L.c2[g];
  }
  for (int g = L.G; g < 10; ++g) out->wg[g] = out->x2g[g] = 0.0;
  return 0;
}

// ---------------------------------------------------------------------------
// General Hermite quadrature on an integer velocity set (the construction the
// paper applies to D2Q37 and D3Q107, for any symmetric set of groups)
// ---------------------------------------------------------------------------
namespace {

struct GenSet {
  int D = 0, G = 0, Q = 0;
  std::vector<std::array<int, 3>> c;  // velocities
  std::vector<int> grp;
};

bool enumerate_set(int D, int G, const int* reps, GenSet* out) {
  out->D = D;
  out->G = G;
  int M = 0;
  for (int g = 0; g < G; ++g)
    for (int a = 0; a < D; ++a) M = std::max(M, std::abs(reps[g * D + a]));
  const int zr = (D == 3) ? M : 0, yr = (D >= 2) ? M : 0;
  for (int g = 0; g < G; ++g) {
    int rep[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) rep[a] = std::abs(reps[g * D + a]);
    std::sort(rep, rep + 3, std::greater<int>());
    int count = 0;
    for (int x = -M; x <= M; ++x)
      for (int y = -yr; y <= yr; ++y)
        for (int z = -zr; z <= zr; ++z) {
          int v[3] = {std::abs(x), std::abs(y), std::abs(z)};
          std::sort(v, v + 3, std::greater<int>());
          if (v[0] != rep[0] || v[1] != rep[1] || v[2] != rep[2]) continue;
          out->c.push_back({x, y, z});
          out->grp.push_back(g);
          ++count;
        }
    if (count == 0) return false;
  }
  out->Q = (int)out->c.size();
  return true;
}

double gen_group_moment(const GenSet& S, int g, const int* alpha, double r) {
  double s = 0.0;
  for (int i = 0; i < S.Q; ++i) {
    if (S.grp[i] != g) continue;
    double m = 1.0;
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < alpha[a]; ++k) m *= r * S.c[i][a];
    s += m;
  }
  return s;
}

// weights for fixed r from all conditions except `drop`; residual of `drop`
bool gen_weights(const GenSet& S, const std::vector<std::array<int, 3>>& cond, int drop, double r, double* w,
                 double* resid) {
  const int G = S.G;
  std::vector<double> a(G * G), b(G);
  int row = 0;
  for (int k = 0; k < (int)cond.size(); ++k) {
    if (k == drop) continue;
    for (int g = 0; g < G; ++g) a[row * G + g] = gen_group_moment(S, g, cond[k].data(), r);
    b[row] = target(cond[k].data());
    ++row;
  }
  if (row != G || !lu_solve(G, a.data(), b.data())) return false;
  for (int g = 0; g < G; ++g) w[g] = b[g];
  if (resid) {
    *resid = 0.0;
    if (drop >= 0) {
      double s = 0.0;
      for (int g = 0; g < G; ++g) s += w[g] * gen_group_moment(S, g, cond[drop].data(), r);
      *resid = s - target(cond[drop].data());
    }
  }
  return true;
}

}  // namespace

int hermite_quadrature(int D, int G, const int* reps, int nconds, const int* exps, double r_in, int* Q,
                       double* w, double* r_out, double* max_residual) {
  if (D < 1 || D > 3 || G < 1 || G > 64 || nconds < 1 || !reps || !exps || !w || !(r_in > 0.0)) return -1;
  GenSet S;
  if (!enumerate_set(D, G, reps, &S)) return -2;
  std::vector<std::array<int, 3>> cond(nconds);
  for (int k = 0; k < nconds; ++k) {
    cond[k] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
      if (exps[k * D + a] < 0 || exps[k * D + a] % 2) return -1;  // even moment classes only
      cond[k][a] = exps[k * D + a];
    }
  }
  double r = r_in;
  std::vector<double> ww(G);
  if (nconds == G) {
    if (!gen_weights(S, cond, -1, r, ww.data(), nullptr)) return -3;
  } else if (nconds == G + 1) {
    // r unknown: drop one condition (the highest-degree one that leaves a
    // regular linear system), solve w(r), and find r by the secant method
    std::vector<int> order(nconds);
    for (int k = 0; k < nconds; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
      return cond[p][0] + cond[p][1] + cond[p][2] > cond[q][0] + cond[q][1] + cond[q][2];
    });
    bool ok = false;
    for (int drop : order) {
      double r0 = r_in * 0.995, r1 = r_in * 1.005, f0, f1;
      if (!gen_weights(S, cond, drop, r0, ww.data(), &f0) || !gen_weights(S, cond, drop, r1, ww.data(), &f1))
        continue;
      for (int it = 0; it < 200 && f1 != f0; ++it) {
        const double r2 = r1 - f1 * (r1 - r0) / (f1 - f0);
        if (!(r2 > 0.0)) break;
        r0 = r1;
        f0 = f1;
        r1 = r2;
        if (!gen_weights(S, cond, drop, r1, ww.data(), &f1)) break;
        if (std::fabs(r1 - r0) <= 1e-16 * r1) break;
      }
      if (gen_weights(S, cond, drop, r1, ww.data(), &f1) && std::fabs(f1) < 1e-9) {
        r = r1;
        ok = true;
        break;
      }
    }
    if (!ok) return -4;
  } else {
    return -5;  // need as many conditions as unknowns
  }
  double worst = 0.0;
  for (int k = 0; k < nconds; ++k) {
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += ww[g] * gen_group_moment(S, g, cond[k].data(), r);
    worst = std::max(worst, std::fabs(s - target(cond[k].data())) / std::max(1.0, target(cond[k].data())));
  }
  for (int g = 0; g < G; ++g) w[g] = ww[g];
  if (Q) *Q = S.Q;
  if (r_out) *r_out = r;
  if (max_residual) *max_residual = worst;
  return 0;
}

// The refinement depends only on the lattice: it is solved once per lattice
// per process, and every instance, pool submission and no-allocation
// reduction copies the result.
int build_lattice_table(int lattice, LatticeTable* out) {
  if (lattice != 0 && lattice != 1) return -1;
  static std::once_flag once[2];
  static LatticeTable table[2];
  static int status[2];
  std::call_once(once[lattice], [lattice] { status[lattice] = build_lattice_table_uncached(lattice, &table[lattice]); });
  if (status[lattice] == 0) *out = table[lattice];
  return status[lattice];
}

}  // namespace lbm
