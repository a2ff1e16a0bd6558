// Slab decomposition of one grid along its slowest axis (host-side plan,
// pack and unpack).
//
// A step pulls every population from at most 3 cells away per axis (the
// integer velocities of Tables I/II have |c_a| <= 3).  A grid split into
// slabs of whole layers along its slowest axis (y in 2D, z in 3D) therefore
// steps exactly like the whole grid if each slab carries 3 ghost layers on
// each side, refreshed before every step with the neighbour's boundary
// layers.  Only the populations that cross the face are needed: ghost layer
// begin - k (k = 1..3) is read only by velocities with c_axis >= k, and
// ghost layer end + k - 1 only by velocities with c_axis <= -k.  At a
// zero-gradient end the ghost layers repeat the edge layer (the clamped
// pull of a single grid).
//
// The plan works on the raw FP64 state layout of lbm_get_state: 2Q planes
// (g for velocities 0..Q-1 in the library's order, then h) of plane_stride
// values, cell index x + nx (y + ny z) of the rank's local grid (its owned
// layers plus the ghost layers).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lattice.h"

namespace lbm {

// Records msg as this thread's lbm_last_error() and returns code (lbm_api.cu).
int set_error(int code, const std::string& msg);

namespace {

constexpr int kGhost = 3;

const LatticeDef& lattice_def(int lattice) { return lattice == LBM_D2Q37 ? kD2Q37 : kD3Q107; }

// velocities whose component along `axis` is >= k (side +1) or <= -k (side -1)
std::vector<int> crossing(const LatticeDef& L, int axis, int side, int k) {
  std::vector<int> v;
  for (int i = 0; i < L.Q; ++i) {
    const int c = L.c[i][axis];
    if ((side > 0 && c >= k) || (side < 0 && c <= -k)) v.push_back(i);
  }
  return v;
}

long long local_layers(const lbm_slab* s) { return (long long)(s->end - s->begin) + 2 * kGhost; }

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" int lbm_slab_plan(int lattice, const int n[3], int periodic, int nranks, int rank, lbm_slab* out) {
  if (lattice != LBM_D2Q37 && lattice != LBM_D3Q107) return set_error(LBM_EINVAL, "unknown lattice");
  if (!n || !out) return set_error(LBM_EINVAL, "n and out must not be NULL");
  if (nranks < 1 || rank < 0 || rank >= nranks) return set_error(LBM_EINVAL, "rank must be in [0, nranks)");
  const int D = (lattice == LBM_D2Q37) ? 2 : 3;
  const int axis = D - 1;
  if (n[0] < 1 || n[1] < 1 || n[2] < 1 || (D == 2 && n[2] != 1))
    return set_error(LBM_EINVAL, "grid dimensions must be positive (nz = 1 for D2Q37)");
  const long long layers = n[axis];
  const long long b = layers * rank / nranks, e = layers * (rank + 1) / nranks;
  // a neighbour's 3 boundary layers must lie on that neighbour alone
  for (int r = 0; r < nranks; ++r)
    if (layers * (r + 1) / nranks - layers * r / nranks < kGhost)
      return set_error(LBM_EINVAL, "every slab needs at least 3 layers (too many ranks for the grid)");
  lbm_slab s{};
  s.lattice = lattice;
  s.axis = axis;
  for (int a = 0; a < 3; ++a) s.n[a] = n[a];
  s.periodic = periodic ? 1 : 0;
  s.nranks = nranks;
  s.rank = rank;
  s.begin = (int)b;
  s.end = (int)e;
  s.lo = (rank > 0) ? rank - 1 : (periodic ? nranks - 1 : -1);
  s.hi = (rank < nranks - 1) ? rank + 1 : (periodic ? 0 : -1);
  s.layer_cells = (D == 2) ? n[0] : n[0] * n[1];
  for (int a = 0; a < 3; ++a) s.local_n[a] = n[a];
  s.local_n[axis] = (int)(e - b) + 2 * kGhost;
  const LatticeDef& L = lattice_def(lattice);
  long long vals = 0;
  for (int k = 1; k <= kGhost; ++k) vals += 2LL * (long long)crossing(L, axis, +1, k).size() * s.layer_cells;
  s.msg_values = vals;  // the same for both sides (the set is symmetric)
  *out = s;
  return LBM_OK;
}

// to_hi: for k = 1..3, owned layer end - k (local layer 3 + nloc - k) of the
// velocities with c_axis >= k, g planes then h planes; to_lo: owned layer
// begin + k - 1 (local layer 3 + k - 1) of the velocities with c_axis <= -k.
extern "C" int lbm_slab_pack(const lbm_slab* s, const double* state, long long plane_stride, double* to_lo,
                             double* to_hi) {
  if (!s || !state) return set_error(LBM_EINVAL, "slab and state must not be NULL");
  const LatticeDef& L = lattice_def(s->lattice);
  const long long lc = s->layer_cells;
  const long long nloc = s->end - s->begin;
  if (plane_stride < local_layers(s) * lc) return set_error(LBM_EINVAL, "plane_stride below the local grid's cells");
  long long o_lo = 0, o_hi = 0;
  for (int k = 1; k <= kGhost; ++k) {
    const long long top = (kGhost + nloc - k) * lc, bottom = (kGhost + k - 1) * lc;
    for (int half = 0; half < 2; ++half) {  // g planes, then h planes
      const long long pofs = (long long)half * L.Q;
      if (to_hi)
        for (int i : crossing(L, s->axis, +1, k)) {
          std::memcpy(to_hi + o_hi, state + (pofs + i) * plane_stride + top, sizeof(double) * lc);
          o_hi += lc;
        }
      if (to_lo)
        for (int i : crossing(L, s->axis, -1, k)) {
          std::memcpy(to_lo + o_lo, state + (pofs + i) * plane_stride + bottom, sizeof(double) * lc);
          o_lo += lc;
        }
    }
  }
  return LBM_OK;
}

// from_lo (the lower neighbour's to_hi) into ghost layers 3 - k, from_hi
// (the upper neighbour's to_lo) into ghost layers 3 + nloc + k - 1.  A side
// without a neighbour (zero-gradient end) copies its edge layer into its
// ghost layers, every plane.
extern "C" int lbm_slab_unpack(const lbm_slab* s, double* state, long long plane_stride, const double* from_lo,
                               const double* from_hi) {
  if (!s || !state) return set_error(LBM_EINVAL, "slab and state must not be NULL");
  const LatticeDef& L = lattice_def(s->lattice);
  const long long lc = s->layer_cells;
  const long long nloc = s->end - s->begin;
  if (plane_stride < local_layers(s) * lc) return set_error(LBM_EINVAL, "plane_stride below the local grid's cells");
  if ((s->lo >= 0 && !from_lo) || (s->hi >= 0 && !from_hi))
    return set_error(LBM_EINVAL, "a message from an existing neighbour is NULL");
  long long o_lo = 0, o_hi = 0;
  for (int k = 1; k <= kGhost; ++k) {
    const long long glo = (kGhost - k) * lc, ghi = (kGhost + nloc + k - 1) * lc;
    for (int half = 0; half < 2; ++half) {
      const long long pofs = (long long)half * L.Q;
      if (s->lo >= 0)
        for (int i : crossing(L, s->axis, +1, k)) {
          std::memcpy(state + (pofs + i) * plane_stride + glo, from_lo + o_lo, sizeof(double) * lc);
          o_lo += lc;
        }
      if (s->hi >= 0)
        for (int i : crossing(L, s->axis, -1, k)) {
          std::memcpy(state + (pofs + i) * plane_stride + ghi, from_hi + o_hi, sizeof(double) * lc);
          o_hi += lc;
        }
    }
  }
  // zero-gradient ends: the ghost layers repeat the edge layer
  for (int p = 0; p < 2 * L.Q; ++p) {
    double* plane = state + (long long)p * plane_stride;
    for (int k = 1; k <= kGhost; ++k) {
      if (s->lo < 0) std::memcpy(plane + (kGhost - k) * lc, plane + kGhost * lc, sizeof(double) * lc);
      if (s->hi < 0)
        std::memcpy(plane + (kGhost + nloc + k - 1) * lc, plane + (kGhost + nloc - 1) * lc, sizeof(double) * lc);
    }
  }
  return LBM_OK;
}
