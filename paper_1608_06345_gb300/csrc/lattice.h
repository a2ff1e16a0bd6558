// Velocity sets of the paper's Tables I (D2Q37) and II (D3Q107), fixed at
// compile time so that the step kernel's direction loop unrolls into
// constant offsets and constant multipliers.
//
// Order: velocity 0 is the rest velocity; then, group by group, pairs
// (c, -c) at indices (2k+1, 2k+2), c being the member of the pair whose
// first non-zero component is positive.  Pairing lets the equilibrium be
// evaluated as the even and odd parts of a polynomial in s = xi.u.
#pragma once

namespace lbm {

struct LatticeDef {
  int D, Q, G;
  int c[107][3];
  int grp[107];
  int rep[10][3];    // group representative: sorted |c| components
  int c2[10];        // |c|^2 of each group
  int members[10];
};

constexpr int kD2Groups[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {2, 0, 0},
                                 {2, 1, 0}, {3, 0, 0}, {3, 1, 0}, {3, 3, 0}};
constexpr int kD3Groups[10][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {1, 1, 1}, {2, 0, 0},
                                  {2, 1, 1}, {2, 2, 0}, {2, 2, 2}, {3, 0, 0}, {3, 1, 1}};

constexpr int cabs(int a) { return a < 0 ? -a : a; }

constexpr bool matches(const int* v, const int* rep) {
  int a[3] = {cabs(v[0]), cabs(v[1]), cabs(v[2])};
  for (int p = 0; p < 3; ++p)
    for (int q = p + 1; q < 3; ++q)
      if (a[q] > a[p]) {
        int t = a[p];
        a[p] = a[q];
        a[q] = t;
      }
  return a[0] == rep[0] && a[1] == rep[1] && a[2] == rep[2];
}

constexpr bool leading_positive(const int* v) {
  for (int k = 0; k < 3; ++k) {
    if (v[k] > 0) return true;
    if (v[k] < 0) return false;
  }
  return false;
}

constexpr LatticeDef make_lattice(int D) {
  LatticeDef L{};
  L.D = D;
  L.G = (D == 2) ? 8 : 10;
  for (int g = 0; g < L.G; ++g) {
    for (int k = 0; k < 3; ++k) L.rep[g][k] = (D == 2) ? kD2Groups[g][k] : kD3Groups[g][k];
    L.c2[g] = L.rep[g][0] * L.rep[g][0] + L.rep[g][1] * L.rep[g][1] + L.rep[g][2] * L.rep[g][2];
    L.members[g] = 0;
  }
  int q = 0;
  const int zr = (D == 3) ? 3 : 0;
  for (int g = 0; g < L.G; ++g) {
    for (int x = -3; x <= 3; ++x)
      for (int y = -3; y <= 3; ++y)
        for (int z = -zr; z <= zr; ++z) {
          int v[3] = {x, y, z};
          if (!matches(v, L.rep[g])) continue;
          if (g == 0) {
            L.c[q][0] = 0; L.c[q][1] = 0; L.c[q][2] = 0;
            L.grp[q] = 0;
            ++q;
            L.members[0] = 1;
            continue;
          }
          if (!leading_positive(v)) continue;
          L.c[q][0] = x; L.c[q][1] = y; L.c[q][2] = z;
          L.c[q + 1][0] = -x; L.c[q + 1][1] = -y; L.c[q + 1][2] = -z;
          L.grp[q] = g;
          L.grp[q + 1] = g;
          q += 2;
          L.members[g] += 2;
        }
  }
  L.Q = q;
  return L;
}

constexpr LatticeDef kD2Q37 = make_lattice(2);
constexpr LatticeDef kD3Q107 = make_lattice(3);

static_assert(kD2Q37.Q == 37, "D2Q37 must have 37 velocities");
static_assert(kD3Q107.Q == 107, "D3Q107 must have 107 velocities");
static_assert(kD2Q37.members[4] == 8 && kD2Q37.members[6] == 8,
              "Perm(2r,r) and Perm(3r,r) have 8 members each");

// FP64 lattice table built on the host (lattice_table.cpp).
struct LatticeTable {
  int D, Q, G;
  double r;          // scaling factor, xi_i = r c_i
  double wg[10];     // weight per group
  double x2g[10];    // |xi|^2 per group = r^2 |c|^2
};

// Builds the refined table; returns 0 on success.
int build_lattice_table(int lattice, LatticeTable* out);

// General Hermite quadrature on the integer velocity set spanned by G group
// representatives (reps[G*D], all sign flips and axis permutations of each):
// weights per group w[G] and scale r such that sum_i w_i (r c_i)^alpha equals
// the unit-Gaussian moment for each of the nconds even monomial classes
// exps[nconds*D].  nconds == G: r = r_in is kept; nconds == G + 1: r is
// solved from r_in.  Returns 0, or a negative code.
int hermite_quadrature(int D, int G, const int* reps, int nconds, const int* exps, double r_in, int* Q,
                       double* w, double* r_out, double* max_residual);

}  // namespace lbm
