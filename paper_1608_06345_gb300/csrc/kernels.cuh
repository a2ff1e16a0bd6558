// Device code of the fused pull-stream + BGK-collide step and its helpers.
//
// Per cell and time step (paper: Eq. (13)-(18), Tables I/II, Sec. V):
//   a1 pull     g~_i(x) = g*_i(x - c_i), h~_i(x) = h*_i(x - c_i)
//   a2 moments  rho = sum g~, rho u = sum xi g~, rho E = sum xi^2/2 g~ + sum h~,
//               T = (2E - u^2) / (D + delta)
//   a3 F_i      w_i rho [A0 + A1 s + A2 s^2 + s^3/6 + s^4/24], s = xi_i.u, the
//               fourth-order Hermite equilibrium of Eq. (18) regrouped in
//               powers of s; A0..A2 depend on the velocity group only, so a
//               (c, -c) pair shares the even part and flips the odd part.
//   a4 Fh_i     (delta/2) T F_i
//   a5 relax    g* = g~ + (F - g~)/tau_f,  h* = h~ + (Fh - h~)/tau_g; store.
//
// Representation: every population is held as its deviation from a fixed
// reference equilibrium of the instance, g_i = gref_i + dg_i with
// gref_i = F_i(rho0, u = 0, T0) and h_i = href_i + dh_i with
// href_i = (delta/2) T0 gref_i.  This is an exact change of variables (the
// scheme is linear in g, h given the moments, and the reference totals are
// known: sum gref = rho0, sum xi gref = 0, sum xi^2/2 gref = rho0 D T0 / 2,
// sum href = rho0 delta T0 / 2).  Working on the small dg, dh keeps FP32 and
// 16-bit storage from losing the momentum to cancellation in sum xi_i g_i.
//
// Storage: structure of arrays, cell index x + nx*(y + ny*z).  FP64/FP32:
// 2Q planes (0..Q-1 for g, Q..2Q-1 for h) of ps elements holding dg, dh.
// 16-bit: Q planes of ps 32-bit pairs, g_i in the low half and h_i in the
// high half, holding dg/gref and dh/hscale.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "lattice.h"

namespace lbm {

constexpr int kPeriodic = 0;
constexpr int kZeroGradient = 1;

// ---------------------------------------------------------------------------
// compile-time helpers
// ---------------------------------------------------------------------------
template <int N, int I = 0, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<N, I + 1>(f);
  }
}

template <int LAT>
struct Lat {
  static constexpr int D = (LAT == 0) ? 2 : 3;
  static constexpr int Q = (LAT == 0) ? 37 : 107;
  static constexpr int G = (LAT == 0) ? 8 : 10;
  __host__ __device__ static constexpr int cx(int i) { return (LAT == 0 ? kD2Q37 : kD3Q107).c[i][0]; }
  __host__ __device__ static constexpr int cy(int i) { return (LAT == 0 ? kD2Q37 : kD3Q107).c[i][1]; }
  __host__ __device__ static constexpr int cz(int i) { return (LAT == 0 ? kD2Q37 : kD3Q107).c[i][2]; }
  __host__ __device__ static constexpr int grp(int i) { return (LAT == 0 ? kD2Q37 : kD3Q107).grp[i]; }
  __host__ __device__ static constexpr int c2(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }
};

// ---------------------------------------------------------------------------
// per-instance constants, already converted to the compute type C on the host
// (a double->float conversion runs on the FP64 pipe, which is slow on GB300)
// ---------------------------------------------------------------------------
template <class C>
struct Args {
  int n[3];          // nx, ny, nz
  int bc[3];         // kPeriodic / kZeroGradient per axis
  long long ps;      // plane stride in elements
  C r;               // xi = r c
  C half_r2;         // r^2 / 2
  C Dd;              // D + delta
  C inv_Dd;          // 1 / (D + delta)
  C half_delta;      // delta / 2
  C omega_f;         // 1 / tau_f
  C omega_g;         // 1 / tau_g
  C rho0, T0, t0;    // reference state; t0 = T0 - 1
  C wg[10];          // group weights
  C x2g[10];         // group |xi|^2
  C gref[10];        // reference equilibrium per group, w rho0 A0(u = 0, t0)
  C pref[10];        // A0(u = 0, t0) - 1 per group
  // 16-bit storage codec: dg = gref * d, dh = hscale * e
  C inv_gref[10], hscale[10], inv_hscale[10];
  unsigned int* flag;  // error word: bit 0 = non-finite rho or T met
};

// ---------------------------------------------------------------------------
// storage codec
// ---------------------------------------------------------------------------
template <class S>
struct IsS16 : std::integral_constant<bool, std::is_same<S, __half>::value ||
                                              std::is_same<S, __nv_bfloat16>::value> {};

template <class S>
__device__ __forceinline__ S ldg_s(const S* p) {
  if constexpr (std::is_same<S, __half>::value) {
    unsigned short v = __ldg(reinterpret_cast<const unsigned short*>(p));
    return __ushort_as_half(v);
  } else if constexpr (std::is_same<S, __nv_bfloat16>::value) {
    unsigned short v = __ldg(reinterpret_cast<const unsigned short*>(p));
    return __ushort_as_bfloat16(v);
  } else {
    return __ldg(p);
  }
}

template <class S>
__device__ __forceinline__ float s16_to_f(S v) {
  if constexpr (std::is_same<S, __half>::value) return __half2float(v);
  else return __bfloat162float(v);
}

template <class S>
__device__ __forceinline__ S f_to_s16(float v) {
  if constexpr (std::is_same<S, __half>::value) return __float2half_rn(v);
  else return __float2bfloat16_rn(v);
}

// decode a stored population of group g into its deviation (dg or dh);
// IS_H selects the h codec
template <class S, class C, bool IS_H>
__device__ __forceinline__ C decode(S v, int g, const Args<C>& a) {
  if constexpr (IsS16<S>::value) {
    const C d = static_cast<C>(s16_to_f(v));
    return IS_H ? a.hscale[g] * d : a.gref[g] * d;
  } else {
    return static_cast<C>(v);
  }
}

template <class S, class C, bool IS_H>
__device__ __forceinline__ S encode(C v, int g, const Args<C>& a) {
  if constexpr (IsS16<S>::value) {
    const C d = IS_H ? v * a.inv_hscale[g] : v * a.inv_gref[g];
    return f_to_s16<S>(static_cast<float>(d));
  } else {
    return static_cast<S>(v);
  }
}

// ---------------------------------------------------------------------------
// population addressing
//   FP64 / FP32 storage: plane p (0..Q-1 for g, Q..2Q-1 for h), element
//     p * ps + cell;
//   16-bit storage: g_i and h_i of a cell are adjacent, one 32-bit pair
//     (g in the low half): plane i holds ps pairs, pair i * ps + cell.  One
//     access moves both populations of a direction.
// ---------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ void unpack16(unsigned v, float& lo, float& hi) {
  if constexpr (std::is_same<S, __half>::value) {
    lo = __half2float(__ushort_as_half((unsigned short)(v & 0xffffu)));
    hi = __half2float(__ushort_as_half((unsigned short)(v >> 16)));
  } else {  // bfloat16: the upper 16 bits of an FP32
    lo = __uint_as_float(v << 16);
    hi = __uint_as_float(v & 0xffff0000u);
  }
}

template <class S>
__device__ __forceinline__ unsigned pack16(float lo, float hi) {
  if constexpr (std::is_same<S, __half>::value)
    return (unsigned)__half_as_ushort(__float2half_rn(lo)) | ((unsigned)__half_as_ushort(__float2half_rn(hi)) << 16);
  else
    return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

// raw stored (g_i, h_i) of a cell (16-bit: the stored relative deviations)
template <int Q, class S, class C>
__device__ __forceinline__ void ld_gh(const S* __restrict__ src, int i, long long ps, size_t cell, C& g, C& h) {
  if constexpr (IsS16<S>::value) {
    float lo, hi;
    unpack16<S>(__ldg(reinterpret_cast<const unsigned*>(src) + ((size_t)i * ps + cell)), lo, hi);
    g = static_cast<C>(lo);
    h = static_cast<C>(hi);
  } else {
    g = static_cast<C>(__ldg(src + ((size_t)i * ps + cell)));
    h = static_cast<C>(__ldg(src + ((size_t)(Q + i) * ps + cell)));
  }
}

// store raw (g_i, h_i) (already in the stored scale)
template <int Q, class S, class C>
__device__ __forceinline__ void st_gh(S* __restrict__ dst, int i, long long ps, size_t cell, C g, C h) {
  if constexpr (IsS16<S>::value) {
    reinterpret_cast<unsigned*>(dst)[(size_t)i * ps + cell] = pack16<S>(static_cast<float>(g), static_cast<float>(h));
  } else {
    dst[(size_t)i * ps + cell] = static_cast<S>(g);
    dst[(size_t)(Q + i) * ps + cell] = static_cast<S>(h);
  }
}

// deviations (dg, dh) of a stored raw pair of group grp
template <class S, class C>
__device__ __forceinline__ void scale_gh(C& g, C& h, int grp, const Args<C>& a) {
  if constexpr (IsS16<S>::value) {
    g *= a.gref[grp];
    h *= a.hscale[grp];
  }
}

// ---------------------------------------------------------------------------
// equilibrium deviations (Eq. (18), regrouped by powers of s per group)
//
// With u2 = |u|^2, t = T - 1, x2 = |xi|^2 of the group:
//   F_i / (w rho) = A0 + A1 s + A2 s^2 + s^3/6 + s^4/24
//   A0 = 1 + P,  P = -u2/2 + t (x2 - D)/2 + u2^2/8 + t (D + 2 - x2) u2 / 4
//                    + t^2 [x2^2 - 2 (D + 2) x2 + D (D + 2)] / 8
//   A1 = 1 - u2/2 + t (x2 - D - 2)/2
//   A2 = 1/2 - u2/4 + t (x2 - D - 4)/4
// and the deviation from gref = w rho0 (1 + pref):
//   dF_i = w [drho (1 + P) + rho0 (P - pref)] + w rho [A1 s + A2 s^2 + ...]
//   dFh_i = (delta/2) (T dF_i + dT gref_i)
// ---------------------------------------------------------------------------
template <int LAT, class C>
struct EqCoef {
  // per-cell polynomials in the group's x2 (see above); the per-group
  // coefficients are formed just before that group's velocities are emitted
  C pa, pb, pc, be0, be1, ga0, ga1;
  C rho, drho;
  C ur[3];  // r u
  C T, dT;
};

template <int LAT, class C>
__device__ __forceinline__ void eq_coeffs(C drho, const C (&u)[3], C dT, const Args<C>& a, EqCoef<LAT, C>& k) {
  using L = Lat<LAT>;
  constexpr C D = C(L::D);
  k.rho = a.rho0 + drho;
  k.drho = drho;
  k.T = a.T0 + dT;
  k.dT = dT;
  const C t = a.t0 + dT;
  const C u2 = u[0] * u[0] + u[1] * u[1] + (L::D == 3 ? u[2] * u[2] : C(0));
  // P = pa + pb x2 + pc x2^2;  A1 = be0 + be1 x2;  A2 = ga0 + ga1 x2
  k.pa = -C(0.5) * u2 - C(0.5) * D * t + C(0.125) * u2 * u2 + C(0.25) * (D + C(2)) * t * u2 +
         C(0.125) * D * (D + C(2)) * t * t;
  k.pb = C(0.5) * t - C(0.25) * t * u2 - C(0.25) * (D + C(2)) * t * t;
  k.pc = C(0.125) * t * t;
  k.be0 = C(1) - C(0.5) * u2 - C(0.5) * (D + C(2)) * t;
  k.be1 = C(0.5) * t;
  k.ga0 = C(0.5) - C(0.25) * u2 - C(0.25) * (D + C(4)) * t;
  k.ga1 = C(0.25) * t;
  k.ur[0] = a.r * u[0];
  k.ur[1] = a.r * u[1];
  k.ur[2] = L::D == 3 ? a.r * u[2] : C(0);
}

// emit(I, dF_i) for every velocity i of [IB, IE): the rest velocity (when
// IB = 0), then the (c, -c) pairs sharing the even part of the polynomial in
// s.  Velocities are ordered by group, so a group's coefficients c0..c4 are
// formed once, at its first pair in the range, and are dead after its last.
// IB is 0 or odd, IE odd or Q (whole pairs only).
template <int LAT, class C, int IB = 0, int IE = Lat<LAT>::Q, class Emit>
__device__ __forceinline__ void eq_emit(const EqCoef<LAT, C>& k, const Args<C>& a, Emit&& emit) {
  using L = Lat<LAT>;
  C c0, c1, c2, c3, c4;
  auto group = [&](int g) {
    const C x2 = a.x2g[g];
    const C P = fma(x2, fma(x2, k.pc, k.pb), k.pa);
    const C W = a.wg[g] * k.rho;
    c0 = a.wg[g] * fma(k.drho, C(1) + P, a.rho0 * (P - a.pref[g]));
    c1 = W * fma(k.be1, x2, k.be0);
    c2 = W * fma(k.ga1, x2, k.ga0);
    c3 = W * C(1.0 / 6.0);
    c4 = W * C(1.0 / 24.0);
  };
  static_assert((IB == 0 || IB % 2 == 1) && (IE == L::Q || IE % 2 == 1) && IB < IE, "whole pairs only");
  if constexpr (IB == 0) {
    group(0);
    emit(std::integral_constant<int, 0>{}, c0);
  }
  static_for<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (i % 2 == 1 && i >= IB && i < IE) {
      constexpr int g = L::grp(i);
      if constexpr (i == IB || L::grp(i - 1) != g) group(g);
      constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
      C s = C(0);
      if constexpr (cx != 0) s = fma(C(cx), k.ur[0], s);
      if constexpr (cy != 0) s = fma(C(cy), k.ur[1], s);
      if constexpr (cz != 0) s = fma(C(cz), k.ur[2], s);
      const C s2 = s * s;
      const C e = fma(s2, fma(s2, c4, c2), c0);
      const C o = s * fma(s2, c3, c1);
      emit(std::integral_constant<int, i>{}, e + o);
      emit(std::integral_constant<int, i + 1>{}, e - o);
    }
  });
}

// dF and dFh of every velocity (used by the init kernel)
template <int LAT, class C, class Emit>
__device__ __forceinline__ void equilibrium_dev(C drho, const C (&u)[3], C dT, const Args<C>& a, Emit&& emit) {
  using L = Lat<LAT>;
  EqCoef<LAT, C> k;
  eq_coeffs<LAT, C>(drho, u, dT, a, k);
  const C hd = a.half_delta;
  eq_emit<LAT, C>(k, a, [&](auto I, C dF) {
    constexpr int g = L::grp(decltype(I)::value);
    emit(I, dF, hd * fma(k.T, dF, dT * a.gref[g]));
  });
}

// ---------------------------------------------------------------------------
// source coordinate of a pull along one axis (|c| <= 3)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pull_coord(int p, int c, int n, int bc) {
  int q = p - c;
  if (bc == kPeriodic) {
    if (n >= 4) {  // one correction at most
      q = (q < 0) ? q + n : q;
      q = (q >= n) ? q - n : q;
    } else {  // n >= 1 and |c| <= 3: at most three corrections
      while (q < 0) q += n;
      while (q >= n) q -= n;
    }
  } else {
    q = q < 0 ? 0 : (q > n - 1 ? n - 1 : q);
  }
  return q;
}

// ---------------------------------------------------------------------------
// moments of a cell from the deviations (Eq. (14), (15)), taken over the
// (c, -c) pairs: sum and difference of the pair
//   drho = sum dg, rho = rho0 + drho, rho u = r sum c dg,
//   rho E = rho0 (D + delta) T0 / 2 + dK + dH with dK = r^2/2 sum c^2 dg, dH = sum dh,
//   T = (2E - u^2)/(D + delta) = T0 + dT,
//   dT = [2 (dK + dH) - rho u^2 - (D + delta) T0 drho] / (rho (D + delta))
// ---------------------------------------------------------------------------
// SCALED: the accessors return the stored 16-bit values d, e (dg = gref d,
// dh = hscale e); the group scales are folded into the sums' coefficients
// instead of decoding every value.
template <int LAT, class C, bool SCALED, class GetG, class GetH>
__device__ __forceinline__ void moments_raw(GetG&& getg, GetH&& geth, const Args<C>& a, C& drho, C (&u)[3],
                                            C& dT) {
  using L = Lat<LAT>;
  C m, H;
  if constexpr (SCALED) {
    m = a.gref[0] * getg(std::integral_constant<int, 0>{});
    H = a.hscale[0] * geth(std::integral_constant<int, 0>{});
  } else {
    m = getg(std::integral_constant<int, 0>{});
    H = geth(std::integral_constant<int, 0>{});
  }
  C jx = C(0), jy = C(0), jz = C(0), k2 = C(0);
  C s1 = C(1), s2 = C(2), s3 = C(3), sc2 = C(0), sh = C(1);  // group scale times 1, 2, 3, |c|^2; h scale
  static_for<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (i % 2 == 1) {
      constexpr int g = L::grp(i);
      if constexpr (SCALED && L::grp(i - 1) != g) {
        s1 = a.gref[g];
        s2 = C(2) * s1;
        s3 = C(3) * s1;
        sc2 = C(L::c2(i)) * s1;
        sh = a.hscale[g];
      }
      auto mul = [&](int c) -> C {  // the coefficient c * scale for |c| <= 3
        const int ac = c < 0 ? -c : c;
        const C v = ac == 1 ? s1 : (ac == 2 ? s2 : s3);
        return c < 0 ? -v : v;
      };
      const C gp = getg(I), gm = getg(std::integral_constant<int, i + 1>{});
      const C sp = gp + gm, df = gp - gm;
      const C hp = geth(I) + geth(std::integral_constant<int, i + 1>{});
      if constexpr (SCALED) {
        m = fma(s1, sp, m);
        if constexpr (L::cx(i) != 0) jx = fma(mul(L::cx(i)), df, jx);
        if constexpr (L::cy(i) != 0) jy = fma(mul(L::cy(i)), df, jy);
        if constexpr (L::cz(i) != 0) jz = fma(mul(L::cz(i)), df, jz);
        k2 = fma(sc2, sp, k2);
        H = fma(sh, hp, H);
      } else {
        m += sp;
        if constexpr (L::cx(i) != 0) jx = fma(C(L::cx(i)), df, jx);
        if constexpr (L::cy(i) != 0) jy = fma(C(L::cy(i)), df, jy);
        if constexpr (L::cz(i) != 0) jz = fma(C(L::cz(i)), df, jz);
        k2 = fma(C(L::c2(i)), sp, k2);
        H += hp;
      }
    }
  });
  (void)s2;
  (void)s3;
  const C rho = a.rho0 + m;
  const C inv = C(1) / rho;
  drho = m;
  u[0] = a.r * jx * inv;
  u[1] = a.r * jy * inv;
  u[2] = (L::D == 3) ? a.r * jz * inv : C(0);
  const C u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const C dE2 = C(2) * fma(a.half_r2, k2, H);
  dT = (dE2 - rho * u2 - a.Dd * a.T0 * m) * inv * a.inv_Dd;
}

template <int LAT, class C, class GetG, class GetH>
__device__ __forceinline__ void moments_dev(GetG&& getg, GetH&& geth, const Args<C>& a, C& drho, C (&u)[3],
                                            C& dT) {
  moments_raw<LAT, C, false>(getg, geth, a, drho, u, dT);
}

// The sums of moments_raw restricted to the velocities [IB, IE) (whole
// pairs): acc = {sum dg, sum c_x dg, sum c_y dg, sum c_z dg,
// r^2/2 sum c^2 dg + sum dh}.  Summing the parts of a partition gives the
// cell's sums (up to rounding order).
template <int LAT, class C, bool SCALED, int IB, int IE, class GetG, class GetH>
__device__ __forceinline__ void moments_partial(GetG&& getg, GetH&& geth, const Args<C>& a, C (&acc)[5]) {
  using L = Lat<LAT>;
  C m = C(0), H = C(0);
  if constexpr (IB == 0) {
    if constexpr (SCALED) {
      m = a.gref[0] * getg(std::integral_constant<int, 0>{});
      H = a.hscale[0] * geth(std::integral_constant<int, 0>{});
    } else {
      m = getg(std::integral_constant<int, 0>{});
      H = geth(std::integral_constant<int, 0>{});
    }
  }
  C jx = C(0), jy = C(0), jz = C(0), k2 = C(0);
  C s1 = C(1), s2 = C(2), s3 = C(3), sc2 = C(0), sh = C(1);
  static_for<L::Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    if constexpr (i % 2 == 1 && i >= IB && i < IE) {
      constexpr int g = L::grp(i);
      if constexpr (SCALED && (i == IB || L::grp(i - 1) != g)) {
        s1 = a.gref[g];
        s2 = C(2) * s1;
        s3 = C(3) * s1;
        sc2 = C(L::c2(i)) * s1;
        sh = a.hscale[g];
      }
      auto mul = [&](int c) -> C {
        const int ac = c < 0 ? -c : c;
        const C v = ac == 1 ? s1 : (ac == 2 ? s2 : s3);
        return c < 0 ? -v : v;
      };
      const C gp = getg(I), gm = getg(std::integral_constant<int, i + 1>{});
      const C sp = gp + gm, df = gp - gm;
      const C hp = geth(I) + geth(std::integral_constant<int, i + 1>{});
      if constexpr (SCALED) {
        m = fma(s1, sp, m);
        if constexpr (L::cx(i) != 0) jx = fma(mul(L::cx(i)), df, jx);
        if constexpr (L::cy(i) != 0) jy = fma(mul(L::cy(i)), df, jy);
        if constexpr (L::cz(i) != 0) jz = fma(mul(L::cz(i)), df, jz);
        k2 = fma(sc2, sp, k2);
        H = fma(sh, hp, H);
      } else {
        m += sp;
        if constexpr (L::cx(i) != 0) jx = fma(C(L::cx(i)), df, jx);
        if constexpr (L::cy(i) != 0) jy = fma(C(L::cy(i)), df, jy);
        if constexpr (L::cz(i) != 0) jz = fma(C(L::cz(i)), df, jz);
        k2 = fma(C(L::c2(i)), sp, k2);
        H += hp;
      }
    }
  });
  (void)s2;
  (void)s3;
  acc[0] = m;
  acc[1] = jx;
  acc[2] = jy;
  acc[3] = jz;
  acc[4] = fma(a.half_r2, k2, H);
}

// drho, u, dT of a cell from its summed partials (the closing lines of
// moments_raw with dK + dH = acc[4])
template <int LAT, class C>
__device__ __forceinline__ void moments_finish(const C (&acc)[5], const Args<C>& a, C& drho, C (&u)[3], C& dT) {
  using L = Lat<LAT>;
  const C m = acc[0];
  const C rho = a.rho0 + m;
  const C inv = C(1) / rho;
  drho = m;
  u[0] = a.r * acc[1] * inv;
  u[1] = a.r * acc[2] * inv;
  u[2] = (L::D == 3) ? a.r * acc[3] * inv : C(0);
  const C u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  dT = (C(2) * acc[4] - rho * u2 - a.Dd * a.T0 * m) * inv * a.inv_Dd;
}

// ---------------------------------------------------------------------------
// collide one cell given its pulled deviations and store the result:
//   g* = g~ + omega_f (dF - g~)
//   h* = h~ + omega_g (dFh - h~) = (omega_g hd T) dF + (1 - omega_g) h~ + omega_g hd dT gref
// ---------------------------------------------------------------------------
// For 16-bit storage the accessors return the stored d, e and the new values
// are formed directly in the stored scale:
//   d* = d + omega_f (dF / gref - d),  e* = (hA / hs) dF + (1 - omega_g) e + hb gref / hs
// FD: the finite-difference variant of Sec. III, which relaxes the cell's own
// values and subtracts the convection term conv(I) = {c_g, c_h} (in the
// stored scale) from the relaxed values.
// relax_store_k: the relaxation and store of the velocities [IB, IE) of a
// cell whose equilibrium coefficients k (formed from its moments by
// eq_coeffs) are known; cell is the element index within a plane (32 bits:
// below 2^32 cells per instance)
template <int LAT, class S, class C, bool IDX32, bool FD, int IB = 0, int IE = Lat<LAT>::Q, class GetG, class GetH,
          class Conv>
__device__ __forceinline__ void relax_store_k(GetG&& getg, GetH&& geth, Conv&& conv, const Args<C>& a,
                                              const EqCoef<LAT, C>& k, S* __restrict__ dst, long long ps,
                                              unsigned cell) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  constexpr bool SCALED = IsS16<S>::value;
  // IDX32: element index plane * ps + cell in unsigned 32 bits (the caller
  // checked that every element index is below 2^32); else plane base + the
  // cell's byte offset in 64 bits
  char* db = reinterpret_cast<char*>(dst) + (size_t)cell * sizeof(S);
  const size_t pb = (size_t)ps * sizeof(S);
  auto st = [&](int plane, S v) {
    if constexpr (IDX32) dst[(unsigned)plane * (unsigned)ps + cell] = v;
    else *reinterpret_cast<S*>(db + (size_t)plane * pb) = v;
  };
  const C hA = a.omega_g * a.half_delta * k.T;
  const C om1 = C(1) - a.omega_g;
  const C hbs = a.omega_g * a.half_delta * k.dT;
  C ig = C(1), hAs = hA, hbg = C(0);  // per-group: 1/gref, hA/hs, hbs gref/hs (16-bit)
  eq_emit<LAT, C, IB, IE>(k, a, [&](auto I, C dF) {
    constexpr int i = decltype(I)::value;
    constexpr int g = L::grp(i);
    const C gi = getg(I), hi = geth(I);
    if constexpr (SCALED) {
      if constexpr (i == IB || L::grp(i == 0 ? 0 : i - 1) != g) {
        ig = a.inv_gref[g];
        hAs = hA * a.inv_hscale[g];
        hbg = hbs * a.gref[g] * a.inv_hscale[g];
      }
      C dn = fma(a.omega_f, fma(dF, ig, -gi), gi);
      C en = fma(hAs, dF, fma(om1, hi, hbg));
      if constexpr (FD) {
        const auto cv = conv(I);
        dn -= cv.g;
        en -= cv.h;
      }
      // one 32-bit (g_i, h_i) pair
      unsigned* dp = reinterpret_cast<unsigned*>(dst);
      const unsigned pv = pack16<S>(static_cast<float>(dn), static_cast<float>(en));
      if constexpr (IDX32) dp[(unsigned)i * (unsigned)ps + cell] = pv;
      else dp[(size_t)i * ps + cell] = pv;
    } else {
      C gn = fma(a.omega_f, dF - gi, gi);
      C hn = fma(hA, dF, fma(om1, hi, hbs * a.gref[g]));
      if constexpr (FD) {
        const auto cv = conv(I);
        gn -= cv.g;
        hn -= cv.h;
      }
      st(i, static_cast<S>(gn));
      st(Q + i, static_cast<S>(hn));
    }
  });
}

// relax_store_k with the equilibrium coefficients formed from the moments
template <int LAT, class S, class C, bool IDX32, bool FD, int IB = 0, int IE = Lat<LAT>::Q, class GetG, class GetH,
          class Conv>
__device__ __forceinline__ void relax_store(GetG&& getg, GetH&& geth, Conv&& conv, const Args<C>& a, C drho,
                                            const C (&u)[3], C dT, S* __restrict__ dst, long long ps,
                                            unsigned cell) {
  EqCoef<LAT, C> k;
  eq_coeffs<LAT, C>(drho, u, dT, a, k);
  relax_store_k<LAT, S, C, IDX32, FD, IB, IE>(getg, geth, conv, a, k, dst, ps, cell);
}

template <int LAT, class S, class C, bool IDX32, bool FD, class GetG, class GetH, class Conv>
__device__ __forceinline__ void collide_store_impl(GetG&& getg, GetH&& geth, Conv&& conv, const Args<C>& a,
                                                   S* __restrict__ dst, long long ps, unsigned cell) {
  C drho, u[3], dT;
  moments_raw<LAT, C, IsS16<S>::value>(getg, geth, a, drho, u, dT);
  if (!(isfinite(drho) && isfinite(dT))) atomicOr(a.flag, 1u);
  relax_store<LAT, S, C, IDX32, FD>(getg, geth, conv, a, drho, u, dT, dst, ps, cell);
}

template <class C>
struct ConvGH {
  C g, h;
};

// the stream-and-collide form: no convection term
template <int LAT, class S, class C, bool IDX32, class GetG, class GetH>
__device__ __forceinline__ void collide_store(GetG&& getg, GetH&& geth, const Args<C>& a, S* __restrict__ dst,
                                              long long ps, unsigned cell) {
  collide_store_impl<LAT, S, C, IDX32, false>(getg, geth, [](auto) { return ConvGH<C>{C(0), C(0)}; }, a, dst, ps,
                                              cell);
}

// raw value of a stored population in the compute type (16-bit: the stored
// relative deviation, not decoded)
template <class S, class C>
__device__ __forceinline__ C raw_value(S v) {
  if constexpr (IsS16<S>::value) return static_cast<C>(s16_to_f(v));
  else return static_cast<C>(v);
}

// ---------------------------------------------------------------------------
// the fused step of one cell
//   STAGE 0: the 2Q pulled values live in registers (D2Q37)
//   STAGE 1: they are staged in shared memory by 4/8-byte cp.async (D3Q107,
//            FP32/FP64 storage): no registers held while the loads fly
//   STAGE 2: staged in shared memory by plain loads (D3Q107, 16-bit storage)
//   STAGE 3: g in registers, h staged in shared memory by cp.async (D3Q107,
//            FP32/FP64): half the shared memory per cell of STAGE 1
//   STAGE 6: 16-bit storage, the Q pulled (g_i, h_i) pairs held packed in
//            registers (one register per direction, half of STAGE 0's) and
//            unpacked where each pass uses them
//   STAGE 9: 16-bit storage, half the pairs packed in registers and the
//            other half staged in shared memory by cp.async (D3Q107)
// A block covers BX consecutive cells of a row (thread = cell).
// ---------------------------------------------------------------------------
// ROW: the block's row (y, z) lies at least 3 cells from every y and z face,
// so no pull of the row wraps or clamps along y or z: the source row of
// direction i is the cell's own row shifted by -(c_y nx + c_z nx ny), the same
// for every thread.  Only the x part of the pull differs between threads (a
// 7-entry table of byte offsets); plane and row shifts are uniform, and the
// stores address the cell through one per-thread pointer plus the uniform
// plane stride.  The arithmetic is that of the general path.
// UNI (with ROW, any row): the row shift of direction i is not -(c_y nx +
// c_z nx ny) but the block-uniform ysh[c_y + 3] + zsh[c_z + 3], the shifts
// of the pulled row and plane after the y and z rules; the rows within 3
// cells of a y or z face take the ROW path's code with these tables.
template <int LAT, class S, class C, int STAGE, int BX, bool IDX32 = false, bool ROW = false, bool UNI = false>
__device__ __forceinline__ void step_cell(const S* __restrict__ src, S* __restrict__ dst, const Args<C>& a, int x,
                                          int y, int z) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  if (x >= nx) return;
  constexpr size_t E = IsS16<S>::value ? 2 * sizeof(S) : sizeof(S);  // bytes per stored element (pair)
  // source offsets for lattice components c = -3..3 (index c + 3); ROW keeps
  // only xb, the byte offset of the pulled x in the cell's own row
  unsigned xo[ROW ? 1 : 7], yo[ROW ? 1 : 7], zo[ROW ? 1 : 7], xb[ROW ? 7 : 1];
  unsigned ysh[UNI ? 7 : 1], zsh[UNI ? 7 : 1];
  const unsigned rowcell = (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)z);
  if constexpr (UNI) {
    static_assert(ROW && IDX32, "uniform shift tables extend the 32-bit ROW path");
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      ysh[k] = (unsigned)(pull_coord(y, k - 3, ny, a.bc[1]) - y) * (unsigned)nx;
      zsh[k] = (L::D == 3) ? (unsigned)(pull_coord(z, k - 3, nz, a.bc[2]) - z) * ((unsigned)nx * (unsigned)ny) : 0u;
    }
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    if constexpr (ROW) {  // element index of the pulled x in the cell's own row (a byte offset without IDX32)
      xb[k] = (rowcell + (unsigned)pull_coord(x, k - 3, nx, a.bc[0])) * (IDX32 ? 1u : (unsigned)E);
    } else {
      xo[k] = (unsigned)pull_coord(x, k - 3, nx, a.bc[0]);
      yo[k] = (unsigned)pull_coord(y, k - 3, ny, a.bc[1]) * (unsigned)nx;
      zo[k] = (L::D == 3) ? (unsigned)pull_coord(z, k - 3, nz, a.bc[2]) * (unsigned)nx * (unsigned)ny : 0u;
    }
  }
  const unsigned cell = (unsigned)x + rowcell;
  const long long ps = a.ps;
  auto src_off = [&](auto I) -> unsigned {
    constexpr int i = decltype(I)::value;
    if constexpr (ROW) return 0u;  // not used on the ROW path
    else return zo[L::cz(i) + 3] + yo[L::cy(i) + 3] + xo[L::cx(i) + 3];
  };
  // addresses = plane base (uniform across the grid) + per-thread byte
  // offset; g_i and h_i share the offset of direction i
  const char* sb = reinterpret_cast<const char*>(src);
  const size_t pb = (size_t)ps * sizeof(S);
  auto ld = [&](auto I, int plane, size_t offb) -> S {
    return ldg_s(reinterpret_cast<const S*>(sb + (size_t)plane * pb + offb));
  };
  // address of the pulled element of direction I in plane `plane` (pair
  // index for 16-bit storage): IDX32 -- the launcher checked that every
  // element index of the buffer is below 2^32 -- in unsigned 32-bit element
  // arithmetic, else plane base + 64-bit byte offset
  auto pptr = [&](int plane, auto I) -> const char* {
    constexpr int i = decltype(I)::value;
    if constexpr (UNI) {
      const unsigned u = (unsigned)plane * (unsigned)ps + ysh[L::cy(i) + 3] + zsh[L::cz(i) + 3];
      return reinterpret_cast<const char*>(src) + (size_t)(u + xb[L::cx(i) + 3]) * E;
    } else if constexpr (ROW && IDX32) {
      // uniform part plane ps - c_y nx - c_z nx ny plus the thread's x index,
      // in unsigned 32-bit arithmetic: the sum is the element index, below 2^32
      const unsigned u = (unsigned)plane * (unsigned)ps - (unsigned)(L::cy(i) * nx) -
                         (unsigned)(L::cz(i)) * ((unsigned)nx * (unsigned)ny);
      return reinterpret_cast<const char*>(src) + (size_t)(u + xb[L::cx(i) + 3]) * E;
    } else if constexpr (ROW) {
      const long long shift = -((long long)L::cy(i) * nx + (long long)L::cz(i) * nx * ny) * (long long)E;
      return sb + ((long long)plane * ps * (long long)E + shift) + xb[L::cx(i) + 3];
    } else if constexpr (IDX32) {
      return reinterpret_cast<const char*>(src) + (size_t)((unsigned)plane * (unsigned)ps + src_off(I)) * E;
    } else {
      return sb + (size_t)plane * ((size_t)ps * E) + (size_t)src_off(I) * E;
    }
  };
  constexpr bool SIDX32 = IDX32;
  if constexpr (STAGE == 0) {
    C g[Q], h[Q];
    static_for<Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      if constexpr (ROW) {
        if constexpr (IsS16<S>::value) {
          float lo, hi;
          unpack16<S>(__ldg(reinterpret_cast<const unsigned*>(pptr(i, I))), lo, hi);
          g[i] = lo;
          h[i] = hi;
        } else {
          g[i] = raw_value<S, C>(ldg_s(reinterpret_cast<const S*>(pptr(i, I))));
          h[i] = raw_value<S, C>(ldg_s(reinterpret_cast<const S*>(pptr(Q + i, I))));
        }
      } else if constexpr (IsS16<S>::value) {  // one 32-bit pair holds g_i and h_i
        const unsigned* sp = reinterpret_cast<const unsigned*>(src);
        const unsigned v = IDX32 ? __ldg(sp + ((unsigned)i * (unsigned)ps + src_off(I)))
                                 : __ldg(sp + ((size_t)i * ps + src_off(I)));
        float lo, hi;
        unpack16<S>(v, lo, hi);
        g[i] = lo;
        h[i] = hi;
      } else if constexpr (IDX32) {
        const unsigned off = src_off(I);
        g[i] = raw_value<S, C>(ldg_s(src + ((unsigned)i * (unsigned)ps + off)));
        h[i] = raw_value<S, C>(ldg_s(src + ((unsigned)(Q + i) * (unsigned)ps + off)));
      } else {
        const size_t offb = (size_t)src_off(I) * sizeof(S);
        g[i] = raw_value<S, C>(ld(I, i, offb));
        h[i] = raw_value<S, C>(ld(I, Q + i, offb));
      }
    });
    collide_store<LAT, S, C, SIDX32>([&](auto I) { return g[decltype(I)::value]; },
                                     [&](auto I) { return h[decltype(I)::value]; }, a, dst, ps, cell);
  } else if constexpr (STAGE == 6) {
    static_assert(IsS16<S>::value, "packed pairs need 16-bit storage");
    unsigned pr[Q];
    static_for<Q>([&](auto I) {
      pr[decltype(I)::value] = __ldg(reinterpret_cast<const unsigned*>(pptr(decltype(I)::value, I)));
    });
    auto lo = [](unsigned v) -> C {
      float l, h;
      unpack16<S>(v, l, h);
      return static_cast<C>(l);
    };
    auto hi = [](unsigned v) -> C {
      float l, h;
      unpack16<S>(v, l, h);
      return static_cast<C>(h);
    };
    C drho, u[3], dT;
    moments_raw<LAT, C, true>([&](auto I) { return lo(pr[decltype(I)::value]); },
                              [&](auto I) { return hi(pr[decltype(I)::value]); }, a, drho, u, dT);
    if (!(isfinite(drho) && isfinite(dT))) atomicOr(a.flag, 1u);
    // an empty asm that claims to change each pair: the relaxation pass
    // unpacks again instead of the compiler keeping the moments pass's 2Q
    // unpacked values alive (it emits no instruction)
    static_for<Q>([&](auto I) { asm volatile("" : "+r"(pr[decltype(I)::value])); });
    relax_store<LAT, S, C, SIDX32, false>([&](auto I) { return lo(pr[decltype(I)::value]); },
                                         [&](auto I) { return hi(pr[decltype(I)::value]); },
                                         [](auto) { return ConvGH<C>{C(0), C(0)}; }, a, drho, u, dT, dst, ps, cell);
  } else if constexpr (STAGE == 9) {
    // 16-bit storage: the pairs of the first (Q + 1) / 2 directions held
    // packed in registers (as STAGE 6), the others staged in shared memory
    // slots [i - NR][thread] by 4-byte cp.async (as STAGE 3 stages h), so a
    // thread holds about half the registers of STAGE 6
    static_assert(IsS16<S>::value, "packed pairs need 16-bit storage");
    constexpr int NR = (Q + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned* sp = reinterpret_cast<unsigned*>(smem_raw);  // [Q - NR][BX]
    const int t = threadIdx.x;
    unsigned pr[NR];
    static_for<Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      if constexpr (i < NR) {
        pr[i] = __ldg(reinterpret_cast<const unsigned*>(pptr(i, I)));
      } else {
        const unsigned sa = (unsigned)__cvta_generic_to_shared(sp + (i - NR) * BX + t);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(pptr(i, I)));
      }
    });
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    const volatile unsigned* spv = sp;
    auto word = [&](auto I) -> unsigned {
      constexpr int i = decltype(I)::value;
      if constexpr (i < NR) return pr[i];
      else return spv[(i - NR) * BX + t];
    };
    auto lo = [&](auto I) -> C {
      float l, h;
      unpack16<S>(word(I), l, h);
      return static_cast<C>(l);
    };
    auto hi = [&](auto I) -> C {
      float l, h;
      unpack16<S>(word(I), l, h);
      return static_cast<C>(h);
    };
    C drho, u[3], dT;
    moments_raw<LAT, C, true>(lo, hi, a, drho, u, dT);
    if (!(isfinite(drho) && isfinite(dT))) atomicOr(a.flag, 1u);
    // as STAGE 6: the relaxation pass unpacks the held pairs again
    static_for<NR>([&](auto I) { asm volatile("" : "+r"(pr[decltype(I)::value])); });
    relax_store<LAT, S, C, SIDX32, false>(lo, hi, [](auto) { return ConvGH<C>{C(0), C(0)}; }, a, drho, u, dT, dst,
                                         ps, cell);
  } else if constexpr (STAGE == 3) {
    static_assert(sizeof(S) == 4 || sizeof(S) == 8, "cp.async needs 4- or 8-byte elements");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* sh = reinterpret_cast<S*>(smem_raw);  // [Q][BX]: h only
    const int t = threadIdx.x;
    C g[Q];
    static_for<Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      const unsigned sa = (unsigned)__cvta_generic_to_shared(sh + i * BX + t);
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(pptr(Q + i, I)), "n"(sizeof(S)));
      g[i] = static_cast<C>(ldg_s(reinterpret_cast<const S*>(pptr(i, I))));
    });
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    // volatile: the moments pass and the relaxation pass each read h_i from
    // shared memory, so the 107 h values are not all held in registers
    const volatile S* shv = sh;
    collide_store<LAT, S, C, SIDX32>([&](auto I) { return g[decltype(I)::value]; },
                                     [&](auto I) { return static_cast<C>(shv[decltype(I)::value * BX + t]); }, a,
                                     dst, ps, cell);
  } else {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* sg = reinterpret_cast<S*>(smem_raw);  // [2Q][BX]
    const int t = threadIdx.x;
    static_for<Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      if constexpr (STAGE == 1) {
        static_assert(sizeof(S) == 4 || sizeof(S) == 8, "cp.async needs 4- or 8-byte elements");
        const unsigned sa0 = (unsigned)__cvta_generic_to_shared(sg + i * BX + t);
        const unsigned sa1 = (unsigned)__cvta_generic_to_shared(sg + (Q + i) * BX + t);
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa0), "l"(pptr(i, I)), "n"(sizeof(S)));
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa1), "l"(pptr(Q + i, I)),
                     "n"(sizeof(S)));
      } else if constexpr (IsS16<S>::value) {  // the 32-bit (g_i, h_i) pair into slot [i][t]
        reinterpret_cast<unsigned*>(smem_raw)[i * BX + t] = __ldg(reinterpret_cast<const unsigned*>(pptr(i, I)));
      } else {
        sg[i * BX + t] = ldg_s(reinterpret_cast<const S*>(pptr(i, I)));
        sg[(Q + i) * BX + t] = ldg_s(reinterpret_cast<const S*>(pptr(Q + i, I)));
      }
    });
    if constexpr (STAGE == 1) asm volatile("cp.async.wait_all;\n" ::: "memory");
    // each thread reads back only the slots it filled itself; the reads are
    // volatile so that each pass re-reads shared memory instead of holding
    // every staged value in registers
    if constexpr (IsS16<S>::value) {
      const volatile unsigned* sp = reinterpret_cast<const volatile unsigned*>(smem_raw);
      collide_store<LAT, S, C, SIDX32>(
          [&](auto I) {
            float lo, hi;
            unpack16<S>(sp[decltype(I)::value * BX + t], lo, hi);
            return static_cast<C>(lo);
          },
          [&](auto I) {
            float lo, hi;
            unpack16<S>(sp[decltype(I)::value * BX + t], lo, hi);
            return static_cast<C>(hi);
          },
          a, dst, ps, cell);
    } else {
      const volatile S* sgv = sg;
      collide_store<LAT, S, C, SIDX32>(
          [&](auto I) { return raw_value<S, C>(sgv[decltype(I)::value * BX + t]); },
          [&](auto I) { return raw_value<S, C>(sgv[(Q + decltype(I)::value) * BX + t]); }, a, dst, ps, cell);
    }
  }
}

// Rows a launch of k_step covers:
//   kRowsAll:      every row (block (x, y, z)); a block whose row lies 3 or
//                  more cells from every y and z face takes the ROW
//                  addressing (the branch is uniform over the block), the
//                  others, and grids too small to have such rows, the
//                  general one.  One kernel, both code paths.
//   kRowsInterior: only those rows (block (x, y - 3, z - 3)), ROW addressing
//   kRowsBoundary: only the other rows of a 3D grid (block (x, k): the k-th
//                  row of the 3-cell z slabs, then of the 3-cell y slabs of
//                  the interior z), ROW addressing with block-uniform row
//                  shift tables (UNI)
//   kRowsUniform:  block (x, y, z) for every row of a 3D grid, all with the
//                  ROW path's code and block-uniform row shift tables (UNI)
// A 3D grid launches kRowsUniform (FP32 storage) or kRowsInterior then
// kRowsBoundary (16-bit storage), so each kernel carries one code path.
constexpr int kRowsAll = 0, kRowsInterior = 1, kRowsBoundary = 2, kRowsUniform = 3;

__device__ __forceinline__ void boundary_row(int k, int ny, int nz, int& y, int& z) {
  if (k < 6 * ny) {
    const int zz = k / ny;
    z = zz < 3 ? zz : nz - 6 + zz;
    y = k - zz * ny;
  } else {
    const int kk = k - 6 * ny;
    z = 3 + kk / 6;
    const int yy = kk - (kk / 6) * 6;
    y = yy < 3 ? yy : ny - 6 + yy;
  }
}

template <int LAT, class S, class C, int STAGE, int BX, int MINB = 1, bool IDX32 = false, int ROWS = kRowsAll>
__global__ void __launch_bounds__(BX, MINB) k_step(const S* __restrict__ src, S* __restrict__ dst, const Args<C> a) {
  const int x = blockIdx.x * BX + threadIdx.x;
  if constexpr (ROWS == kRowsInterior) {
    step_cell<LAT, S, C, STAGE, BX, IDX32, true>(src, dst, a, x, blockIdx.y + 3, blockIdx.z + 3);
  } else if constexpr (ROWS == kRowsUniform) {
    step_cell<LAT, S, C, STAGE, BX, true, true, true>(src, dst, a, x, blockIdx.y, blockIdx.z);
  } else if constexpr (ROWS == kRowsBoundary) {
    int y, z;
    boundary_row(blockIdx.y, a.n[1], a.n[2], y, z);
    // the ROW path's code with block-uniform row shifts (UNI), where element
    // indices fit 32 bits; else the general path
    if constexpr (IDX32) step_cell<LAT, S, C, STAGE, BX, true, true, true>(src, dst, a, x, y, z);
    else step_cell<LAT, S, C, STAGE, BX, IDX32, false>(src, dst, a, x, y, z);
  } else {
    const int y = blockIdx.y, z = blockIdx.z;
    // (the per-thread byte offsets of the ROW path are 32-bit: N E < 2^32)
    constexpr long long E = IsS16<S>::value ? 2 * (long long)sizeof(S) : (long long)sizeof(S);
    const bool row = y >= 3 && y < a.n[1] - 3 && (Lat<LAT>::D == 2 || (z >= 3 && z < a.n[2] - 3)) &&
                     (long long)a.n[0] * a.n[1] * a.n[2] * E < (1LL << 32);
    if (row)
      step_cell<LAT, S, C, STAGE, BX, IDX32, true>(src, dst, a, x, y, z);
    else
      step_cell<LAT, S, C, STAGE, BX, IDX32, false>(src, dst, a, x, y, z);
  }
}

// ---------------------------------------------------------------------------
// the velocity-split step (STAGE 4): a block of P warps covers 32 cells of a
// row; warp w pulls, sums and relaxes only its part [begin(w), end(w)) of the
// velocities.  The parts' five partial sums meet in shared memory and every
// warp adds them in the same order, so all parts use identical moments.
// Each thread holds 2 (end - begin) values instead of 2Q, which keeps the
// register count near that of the D2Q37 kernel for D3Q107.
// ---------------------------------------------------------------------------
template <int LAT, int P>
struct Split {
  static constexpr int NP = (Lat<LAT>::Q - 1) / 2;  // (c, -c) pairs
  // part 0: the rest velocity and pairs [0, NP/P); part w: pairs [w NP/P, (w+1) NP/P)
  __host__ __device__ static constexpr int begin(int w) { return w == 0 ? 0 : 1 + 2 * (w * NP / P); }
  __host__ __device__ static constexpr int end(int w) { return 1 + 2 * ((w + 1) * NP / P); }
  __host__ __device__ static constexpr int kmax() {
    int m = 0;
    for (int w = 0; w < P; ++w) m = (end(w) - begin(w) > m) ? end(w) - begin(w) : m;
    return m;
  }
};

// SHARE: warp 0 alone finishes the moments and forms the equilibrium
// coefficients, which the other warps read from shared memory after a second
// barrier (less arithmetic per cell; worth it where the FP64 pipe is the bound)
template <int LAT, class S, class C, int P, int MINB, bool SHARE = false>
__global__ void __launch_bounds__(32 * P, MINB) k_step_split(const S* __restrict__ src, S* __restrict__ dst,
                                                            const Args<C> a) {
  using L = Lat<LAT>;
  using SP = Split<LAT, P>;
  constexpr int Q = L::Q;
  constexpr int K = SP::kmax();
  constexpr bool SCALED = IsS16<S>::value;
  __shared__ C red[P][5][32];
  const int lane = threadIdx.x, w = threadIdx.y;
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int x = blockIdx.x * 32 + lane, y = blockIdx.y, z = blockIdx.z;
  const bool active = x < nx;
  const int xs = active ? x : nx - 1;  // lanes past the row end pull from a valid cell and store nothing
  unsigned xo[7], yo[7], zo[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    xo[k] = (unsigned)pull_coord(xs, k - 3, nx, a.bc[0]);
    yo[k] = (unsigned)pull_coord(y, k - 3, ny, a.bc[1]) * (unsigned)nx;
    zo[k] = (L::D == 3) ? (unsigned)pull_coord(z, k - 3, nz, a.bc[2]) * (unsigned)nx * (unsigned)ny : 0u;
  }
  const unsigned cell = (unsigned)xs + (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)z);
  const long long ps = a.ps;
  const char* sb = reinterpret_cast<const char*>(src);
  const size_t pb = (size_t)ps * sizeof(S);
  C g[K], h[K];
  // phase 1: pull this warp's velocities and sum its partial moments
  static_for<P>([&](auto W) {
    constexpr int IB = SP::begin(decltype(W)::value), IE = SP::end(decltype(W)::value);
    if (w == decltype(W)::value) {
      static_for<Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if constexpr (i >= IB && i < IE) {
          const unsigned off = zo[L::cz(i) + 3] + yo[L::cy(i) + 3] + xo[L::cx(i) + 3];
          if constexpr (SCALED) {
            const unsigned v = __ldg(reinterpret_cast<const unsigned*>(src) + ((size_t)i * ps + off));
            float lo, hi;
            unpack16<S>(v, lo, hi);
            g[i - IB] = lo;
            h[i - IB] = hi;
          } else {
            const size_t offb = (size_t)off * sizeof(S);
            g[i - IB] = static_cast<C>(ldg_s(reinterpret_cast<const S*>(sb + (size_t)i * pb + offb)));
            h[i - IB] = static_cast<C>(ldg_s(reinterpret_cast<const S*>(sb + (size_t)(Q + i) * pb + offb)));
          }
        }
      });
      C acc[5];
      moments_partial<LAT, C, SCALED, IB, IE>([&](auto I) { return g[decltype(I)::value - IB]; },
                                              [&](auto I) { return h[decltype(I)::value - IB]; }, a, acc);
#pragma unroll
      for (int k = 0; k < 5; ++k) red[w][k][lane] = acc[k];
    }
  });
  __syncthreads();
  auto finish = [&](EqCoef<LAT, C>& k) {  // sum the parts in a fixed order, then the cell's coefficients
    C acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      C v = red[0][q][lane];
#pragma unroll
      for (int p = 1; p < P; ++p) v += red[p][q][lane];
      acc[q] = v;
    }
    C drho, u[3], dT;
    moments_finish<LAT, C>(acc, a, drho, u, dT);
    if (w == 0 && active && !(isfinite(drho) && isfinite(dT))) atomicOr(a.flag, 1u);
    eq_coeffs<LAT, C>(drho, u, dT, a, k);
  };
  EqCoef<LAT, C> k;
  if constexpr (SHARE) {
    __shared__ EqCoef<LAT, C> shk[32];
    if (w == 0) {
      finish(k);
      shk[lane] = k;
    }
    __syncthreads();
    if (w != 0) k = shk[lane];
  } else {
    finish(k);
  }
  if (!active) return;
  // phase 2: relax and store this warp's velocities
  static_for<P>([&](auto W) {
    constexpr int IB = SP::begin(decltype(W)::value), IE = SP::end(decltype(W)::value);
    if (w == decltype(W)::value)
      relax_store_k<LAT, S, C, false, false, IB, IE>(
          [&](auto I) { return g[decltype(I)::value - IB]; }, [&](auto I) { return h[decltype(I)::value - IB]; },
          [](auto) { return ConvGH<C>{C(0), C(0)}; }, a, k, dst, ps, cell);
  });
}

// ---------------------------------------------------------------------------
// the mirror-pair step (STAGE 8): every cell is worked by two lanes of one
// warp, lane l and lane l ^ 16.  The lower half-warp (half 0, sign +1) takes
// the member c of each (c, -c) pair and the rest velocity; the upper half
// (half 1, sign -1) takes the member -c.  Both halves run one instruction
// stream:
//   - the pull of -c reads x + c, so the sign is folded into the 7-entry
//     offset tables of each axis, and the member -c lies one plane after c;
//   - s(-c; u) = s(c; -u): with u negated the pair's even part e(s^2) is the
//     same and the odd part flips, so each half stores e + o with its own
//     sign of u;
//   - the five moment sums of the halves meet by one __shfl_xor_sync each;
//     both lanes add (or subtract) the two halves' partial sums in the same
//     operand order, so they hold bitwise identical moments.
// A thread holds the (Q + 1) / 2 pulled (g, h) of its half instead of Q, so
// about twice the warps fit per SM; the pair's even and odd parts are formed
// by both lanes.  A block of BX threads covers BX / 2 cells of a row; lanes
// past the row end pull from a valid cell, take part in the shuffles and
// store nothing.
// ---------------------------------------------------------------------------
template <int LAT, class S, class C, int BX, int MINB, bool IDX32, bool HS>
__global__ void __launch_bounds__(BX, MINB) k_step_mirror(const S* __restrict__ src, S* __restrict__ dst,
                                                         const Args<C> a) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  constexpr int NP = (Q - 1) / 2;  // (c, -c) pairs; pair k is velocities 2k+1 (c) and 2k+2 (-c)
  constexpr bool SCALED = IsS16<S>::value;
  static_assert(BX % 32 == 0, "whole warps");
  static_assert(!(HS && SCALED), "16-bit pairs are held packed in registers");
  const int lane = threadIdx.x & 31;
  const int half = lane >> 4;
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int x = blockIdx.x * (BX / 2) + (threadIdx.x >> 5) * 16 + (lane & 15);
  const int y = blockIdx.y, z = blockIdx.z;
  const bool active = x < nx;
  const int xs = active ? x : nx - 1;
  const int sg = half ? -1 : 1;
  // source offsets of the pull of sg * c for c = -3..3 (index c + 3)
  unsigned xo[7], yo[7], zo[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    xo[k] = (unsigned)pull_coord(xs, sg * (k - 3), nx, a.bc[0]);
    yo[k] = (unsigned)pull_coord(y, sg * (k - 3), ny, a.bc[1]) * (unsigned)nx;
    zo[k] = (L::D == 3) ? (unsigned)pull_coord(z, sg * (k - 3), nz, a.bc[2]) * (unsigned)nx * (unsigned)ny : 0u;
  }
  const unsigned cell = (unsigned)xs + (unsigned)nx * ((unsigned)y + (unsigned)ny * (unsigned)z);
  const long long ps = a.ps;
  // element index of this half's member in plane `plane` (pair index for
  // 16-bit storage) at cell offset off
  auto eidx = [&](int plane, unsigned off) -> size_t {
    if constexpr (IDX32) return (size_t)((unsigned)(plane + half) * (unsigned)ps + off);
    else return (size_t)(plane + half) * (size_t)ps + off;
  };
  // the pulled values: FP32/FP64 g in registers and h in registers or (HS)
  // in shared memory slots [k][thread] filled by cp.async; 16-bit storage
  // the packed (g, h) pairs in registers.  The rest velocity is pulled by
  // half 0 only (half 1 keeps zeros).
  C g0 = C(0), h0 = C(0);
  C g[SCALED ? 1 : NP];
  C h[(SCALED || HS) ? 1 : NP];
  unsigned pr[SCALED ? NP : 1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* shh = reinterpret_cast<S*>(smem_raw);  // HS: [NP][BX]
  if (half == 0) {
    if constexpr (SCALED) {
      float lo, hi;
      unpack16<S>(__ldg(reinterpret_cast<const unsigned*>(src) + (size_t)cell), lo, hi);
      g0 = lo;
      h0 = hi;
    } else {
      g0 = static_cast<C>(ldg_s(src + (size_t)cell));
      h0 = static_cast<C>(ldg_s(src + (size_t)Q * (size_t)ps + cell));
    }
  }
  static_for<NP>([&](auto K) {
    constexpr int k = decltype(K)::value;
    constexpr int i = 2 * k + 1;
    const unsigned off = zo[L::cz(i) + 3] + yo[L::cy(i) + 3] + xo[L::cx(i) + 3];
    if constexpr (SCALED) {
      pr[k] = __ldg(reinterpret_cast<const unsigned*>(src) + eidx(i, off));
    } else {
      if constexpr (HS) {
        static_assert(sizeof(S) == 4 || sizeof(S) == 8, "cp.async needs 4- or 8-byte elements");
        const unsigned sa = (unsigned)__cvta_generic_to_shared(shh + k * BX + threadIdx.x);
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(src + eidx(Q + i, off)),
                     "n"(sizeof(S)));
      } else {
        h[k] = static_cast<C>(ldg_s(src + eidx(Q + i, off)));
      }
      g[k] = static_cast<C>(ldg_s(src + eidx(i, off)));
    }
  });
  if constexpr (HS) asm volatile("cp.async.wait_all;\n" ::: "memory");
  // accessors of the pulled g, h of pair k (16-bit: the stored relative
  // deviations, unpacked where they are used; HS: h re-read from shared
  // memory by each pass)
  const volatile S* shv = shh;
  auto getg = [&](int k) -> C {
    if constexpr (SCALED) {
      float lo, hi;
      unpack16<S>(pr[k], lo, hi);
      return static_cast<C>(lo);
    } else {
      return g[k];
    }
  };
  auto geth = [&](int k) -> C {
    if constexpr (SCALED) {
      float lo, hi;
      unpack16<S>(pr[k], lo, hi);
      return static_cast<C>(hi);
    } else if constexpr (HS) {
      return static_cast<C>(shv[k * BX + threadIdx.x]);
    } else {
      return h[k];
    }
  };
  // this half's partial sums, with the member c's components (for half 1
  // the momentum sums are minus its share)
  C m, H, jx = C(0), jy = C(0), jz = C(0), k2 = C(0);
  if constexpr (SCALED) {
    m = a.gref[0] * g0;
    H = a.hscale[0] * h0;
  } else {
    m = g0;
    H = h0;
  }
  {
    C s1 = C(1), sc2 = C(0), sh = C(1);
    static_for<NP>([&](auto K) {
      constexpr int k = decltype(K)::value;
      constexpr int i = 2 * k + 1;
      constexpr int gr = L::grp(i);
      const C gk = getg(k), hk = geth(k);
      if constexpr (SCALED) {
        if constexpr (k == 0 || L::grp(i - 2) != gr) {
          s1 = a.gref[gr];
          sc2 = C(L::c2(i)) * s1;
          sh = a.hscale[gr];
        }
        const C gv = s1 * gk;
        m += gv;
        if constexpr (L::cx(i) != 0) jx = fma(C(L::cx(i)), gv, jx);
        if constexpr (L::cy(i) != 0) jy = fma(C(L::cy(i)), gv, jy);
        if constexpr (L::cz(i) != 0) jz = fma(C(L::cz(i)), gv, jz);
        k2 = fma(sc2, gk, k2);
        H = fma(sh, hk, H);
      } else {
        m += gk;
        if constexpr (L::cx(i) != 0) jx = fma(C(L::cx(i)), gk, jx);
        if constexpr (L::cy(i) != 0) jy = fma(C(L::cy(i)), gk, jy);
        if constexpr (L::cz(i) != 0) jz = fma(C(L::cz(i)), gk, jz);
        k2 = fma(C(L::c2(i)), gk, k2);
        H += hk;
      }
    });
    (void)s1;
    (void)sc2;
    (void)sh;
  }
  const C e4 = fma(a.half_r2, k2, H);
  // combine the halves: lower + upper for the even sums, lower - upper for
  // the momentum; both lanes evaluate the same operation on the same operands
  C acc[5];
  {
    const C own[5] = {m, jx, jy, jz, e4};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      if (q == 3 && L::D == 2) {
        acc[q] = C(0);
        continue;
      }
      const C other = __shfl_xor_sync(0xffffffffu, own[q], 16);
      const C lo = half ? other : own[q];
      const C up = half ? own[q] : other;
      acc[q] = (q >= 1 && q <= 3) ? lo - up : lo + up;
    }
  }
  C drho, u[3], dT;
  moments_finish<LAT, C>(acc, a, drho, u, dT);
  if (active && half == 0 && !(isfinite(drho) && isfinite(dT))) atomicOr(a.flag, 1u);
  if constexpr (SCALED) {
    // an empty asm that claims to change each pair: the relaxation pass
    // unpacks again instead of keeping the moments pass's unpacked values
    // alive (it emits no instruction)
    static_for<NP>([&](auto K) { asm volatile("" : "+r"(pr[decltype(K)::value])); });
  }
  EqCoef<LAT, C> kc;
  eq_coeffs<LAT, C>(drho, u, dT, a, kc);
  // this half's sign of u: s of the member -c is s(c) at -u
#pragma unroll
  for (int q = 0; q < 3; ++q) kc.ur[q] = half ? -kc.ur[q] : kc.ur[q];
  // relax and store
  const C hA = a.omega_g * a.half_delta * kc.T;
  const C om1 = C(1) - a.omega_g;
  const C hbs = a.omega_g * a.half_delta * kc.dT;
  auto store = [&](int i, unsigned plane_half, C gn, C hn) {
    // the stored plane is i + plane_half
    if constexpr (SCALED) {
      unsigned* dp = reinterpret_cast<unsigned*>(dst);
      const unsigned pv = pack16<S>(static_cast<float>(gn), static_cast<float>(hn));
      if constexpr (IDX32) dp[(unsigned)(i + plane_half) * (unsigned)ps + cell] = pv;
      else dp[(size_t)(i + plane_half) * ps + cell] = pv;
    } else {
      if constexpr (IDX32) {
        dst[(unsigned)(i + plane_half) * (unsigned)ps + cell] = static_cast<S>(gn);
        dst[(unsigned)(Q + i + plane_half) * (unsigned)ps + cell] = static_cast<S>(hn);
      } else {
        dst[(size_t)(i + plane_half) * ps + cell] = static_cast<S>(gn);
        dst[(size_t)(Q + i + plane_half) * ps + cell] = static_cast<S>(hn);
      }
    }
  };
  // per group: the equilibrium coefficients c0..c4 and the relaxation's
  // constants (ig = 1/gref, hAs = hA/hscale, hbg = hbs gref/hscale for
  // 16-bit storage; hAs = hA, hbg = hbs gref otherwise)
  C c0, c1, c2, c3, c4, ig, hAs, hbg;
  auto group = [&](int gr) {
    const C x2 = a.x2g[gr];
    const C P = fma(x2, fma(x2, kc.pc, kc.pb), kc.pa);
    const C W = a.wg[gr] * kc.rho;
    c0 = a.wg[gr] * fma(kc.drho, C(1) + P, a.rho0 * (P - a.pref[gr]));
    c1 = W * fma(kc.be1, x2, kc.be0);
    c2 = W * fma(kc.ga1, x2, kc.ga0);
    c3 = W * C(1.0 / 6.0);
    c4 = W * C(1.0 / 24.0);
    if constexpr (SCALED) {
      ig = a.inv_gref[gr];
      hAs = hA * a.inv_hscale[gr];
      hbg = hbs * a.gref[gr] * a.inv_hscale[gr];
    } else {
      ig = C(1);
      hAs = hA;
      hbg = hbs * a.gref[gr];
    }
  };
  auto relax = [&](C dF, C gv, C hv, C& gn, C& hn) {
    if constexpr (SCALED) gn = fma(a.omega_f, fma(dF, ig, -gv), gv);
    else gn = fma(a.omega_f, dF - gv, gv);
    hn = fma(hAs, dF, fma(om1, hv, hbg));
  };
  group(0);
  if (active && half == 0) {
    C gn, hn;
    relax(c0, g0, h0, gn, hn);
    store(0, 0u, gn, hn);
  }
  static_for<NP>([&](auto K) {
    constexpr int k = decltype(K)::value;
    constexpr int i = 2 * k + 1;
    constexpr int gr = L::grp(i);
    if constexpr (k == 0 || L::grp(i - 2) != gr) group(gr);
    C s = C(0);
    if constexpr (L::cx(i) != 0) s = fma(C(L::cx(i)), kc.ur[0], s);
    if constexpr (L::cy(i) != 0) s = fma(C(L::cy(i)), kc.ur[1], s);
    if constexpr (L::cz(i) != 0) s = fma(C(L::cz(i)), kc.ur[2], s);
    const C s2 = s * s;
    const C e = fma(s2, fma(s2, c4, c2), c0);
    const C o = s * fma(s2, c3, c1);
    C gn, hn;
    relax(e + o, getg(k), geth(k), gn, hn);
    if (active) store(i, (unsigned)half, gn, hn);
  });
}

// ---------------------------------------------------------------------------
// the finite-difference variant of Sec. III (Eq. (16)/(17) with the
// convection term discretised along each axis by the third-order upwind
// difference; the printed g_j is read as g_i), lamr = lambda r, lambda = dt/dx:
//   q*_i = q_i - lambda xi_i . D(q_i) - omega (q_i - Q_eq,i)
//   D_a(q) at p for c_a > 0: [q(p-2) - 6 q(p-1) + 3 q(p) + 2 q(p+1)] / 6
//                 for c_a < 0: [-q(p+2) + 6 q(p+1) - 3 q(p) - 2 q(p-1)] / 6
// One thread per cell; the own 2Q values in registers, the upwind neighbours
// read per direction (their reuse across the block is served by L1/L2).
// ---------------------------------------------------------------------------
template <int LAT, class S, class C, int BX>
__global__ void __launch_bounds__(BX) k_step_fd(const S* __restrict__ src, S* __restrict__ dst, const Args<C> a,
                                                C lamr) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  const int x = blockIdx.x * BX + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  if (x >= nx) return;
  // positions p + k, k = -2..2 (index k + 2), after the boundary rule
  unsigned xp[5], yp[5], zp[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    xp[k] = (unsigned)pull_coord(x, 2 - k, nx, a.bc[0]);
    yp[k] = (unsigned)pull_coord(y, 2 - k, ny, a.bc[1]) * (unsigned)nx;
    zp[k] = (L::D == 3) ? (unsigned)pull_coord(z, 2 - k, nz, a.bc[2]) * (unsigned)nx * (unsigned)ny : 0u;
  }
  const unsigned cell = xp[2] + yp[2] + zp[2];
  const long long ps = a.ps;
  C g[Q], h[Q];
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    ld_gh<Q, S, C>(src, i, ps, cell, g[i], h[i]);
  });
  // upwind differences of g_i and h_i along one axis with position table
  // `pos` (the other two axes at the cell's own position `rest`)
  auto upwind = [&](int i, int sgn, const unsigned (&pos)[5], unsigned rest, C og, C oh, C& dg, C& dh) {
    C gm2, hm2, gm1, hm1, gp1, hp1;  // values at the upwind-2, upwind-1 and downwind-1 positions
    const int u2 = sgn > 0 ? 0 : 4, u1 = sgn > 0 ? 1 : 3, d1 = sgn > 0 ? 3 : 1;
    ld_gh<Q, S, C>(src, i, ps, pos[u2] + rest, gm2, hm2);
    ld_gh<Q, S, C>(src, i, ps, pos[u1] + rest, gm1, hm1);
    ld_gh<Q, S, C>(src, i, ps, pos[d1] + rest, gp1, hp1);
    const C sg = sgn > 0 ? C(1) : C(-1);
    dg = sg * (gm2 - C(6) * gm1 + C(3) * og + C(2) * gp1) * C(1.0 / 6.0);
    dh = sg * (hm2 - C(6) * hm1 + C(3) * oh + C(2) * hp1) * C(1.0 / 6.0);
  };
  auto conv = [&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
    C cg = C(0), ch = C(0), dg, dh;
    if constexpr (cx != 0) {
      upwind(i, cx, xp, yp[2] + zp[2], g[i], h[i], dg, dh);
      cg = fma(C(cx), dg, cg);
      ch = fma(C(cx), dh, ch);
    }
    if constexpr (cy != 0) {
      upwind(i, cy, yp, xp[2] + zp[2], g[i], h[i], dg, dh);
      cg = fma(C(cy), dg, cg);
      ch = fma(C(cy), dh, ch);
    }
    if constexpr (cz != 0) {
      upwind(i, cz, zp, xp[2] + yp[2], g[i], h[i], dg, dh);
      cg = fma(C(cz), dg, cg);
      ch = fma(C(cz), dh, ch);
    }
    return ConvGH<C>{lamr * cg, lamr * ch};
  };
  collide_store_impl<LAT, S, C, false, true>([&](auto I) { return g[decltype(I)::value]; },
                                             [&](auto I) { return h[decltype(I)::value]; }, conv, a, dst, ps,
                                             cell);
}

// ---------------------------------------------------------------------------
// batched step of a pool of independent instances (continuous batching)
//
// Every resident instance has a slot descriptor in device memory (its
// constants, its two buffers, which buffer is current and how many steps it
// still has to take) and contributes tiles of BX cells along a row to one
// flat tile list.  A persistent grid walks the list; tiles of instances with
// no steps left are skipped.  Each cell runs exactly the arithmetic of the
// single-instance kernel, so an instance's result does not depend on what
// else is resident.  k_pool_advance then decrements the step counters and
// flips the buffers (and stops an instance whose error word is set); a
// bundle of steps is a CUDA graph of these two kernels.
// ---------------------------------------------------------------------------
template <class C>
struct PoolSlot {
  Args<C> a;
  void* buf[2];
  int cur;         // buffer holding the current state
  int steps_left;  // steps still to take
};

template <int LAT, class S, class C, int STAGE, int BX>
__global__ void __launch_bounds__(BX) k_pool_step(const PoolSlot<C>* __restrict__ slots,
                                                  const int4* __restrict__ tiles, const int* __restrict__ n_tiles) {
  const int nt = *n_tiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const int4 tl = tiles[t];  // slot, x0, y, z
    const PoolSlot<C>& sl = slots[tl.x];
    if (sl.steps_left <= 0) continue;
    const int c = sl.cur;
    step_cell<LAT, S, C, STAGE, BX>(static_cast<const S*>(sl.buf[c]), static_cast<S*>(sl.buf[c ^ 1]), sl.a,
                                    tl.y + (int)threadIdx.x, tl.z, tl.w);
  }
}

template <class C>
__global__ void k_pool_advance(PoolSlot<C>* __restrict__ slots, int nslots) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nslots && slots[i].steps_left > 0) {
    if (*slots[i].a.flag) {
      slots[i].steps_left = 0;  // a non-finite instance takes no further steps
    } else {
      slots[i].steps_left -= 1;
      slots[i].cur ^= 1;
    }
  }
}

// ---------------------------------------------------------------------------
// init: g = F(rho, u, T), h = (delta/2) T F from FP64 device fields, stored
// as deviations from the reference equilibrium.  Arithmetic in the compute
// type C of the instance (FP64 only for FP64 instances); the differences
// rho - rho0 and T - T0 are taken in FP64 before rounding to C.
// ---------------------------------------------------------------------------
template <int LAT, class S, class C>
__global__ void k_init(S* __restrict__ dst, const double* __restrict__ rho, const double* __restrict__ u,
                       const double* __restrict__ T, long long N, const Args<C> a, double rho0, double T0) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= N) return;
  const C drho = static_cast<C>(rho[cell] - rho0), dT = static_cast<C>(T[cell] - T0);
  const C uu[3] = {static_cast<C>(u[cell]), static_cast<C>(u[N + cell]),
                   L::D == 3 ? static_cast<C>(u[2 * N + cell]) : C(0)};
  const long long ps = a.ps;
  equilibrium_dev<LAT, C>(drho, uu, dT, a, [&](auto I, C dF, C dFh) {
    constexpr int i = decltype(I)::value;
    if constexpr (IsS16<S>::value)
      st_gh<Q, S, C>(dst, i, ps, cell, dF * a.inv_gref[L::grp(i)], dFh * a.inv_hscale[L::grp(i)]);
    else
      st_gh<Q, S, C>(dst, i, ps, cell, dF, dFh);
  });
}

// ---------------------------------------------------------------------------
// moments of the stored state (rho, u, T out in FP64), arithmetic in the
// compute type C; rho0 + drho and T0 + dT are formed in FP64
// ---------------------------------------------------------------------------
template <int LAT, class S, class C>
__global__ void k_moments(const S* __restrict__ src, double* __restrict__ rho, double* __restrict__ u,
                          double* __restrict__ T, long long N, const Args<C> a, double rho0, double T0) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= N) return;
  const long long ps = a.ps;
  C g[Q], h[Q];
  static_for<Q>([&](auto I) {
    constexpr int i = decltype(I)::value;
    ld_gh<Q, S, C>(src, i, ps, cell, g[i], h[i]);
  });
  C drho, uu[3], dT;
  moments_raw<LAT, C, IsS16<S>::value>([&](auto I) { return g[decltype(I)::value]; },
                                       [&](auto I) { return h[decltype(I)::value]; }, a, drho, uu, dT);
  rho[cell] = rho0 + static_cast<double>(drho);
  u[cell] = static_cast<double>(uu[0]);
  u[N + cell] = static_cast<double>(uu[1]);
  if (L::D == 3) u[2 * N + cell] = static_cast<double>(uu[2]);
  T[cell] = T0 + static_cast<double>(dT);
}

// deviations (dg_i, dh_i) of a cell in double for the FP64 reductions
// (16-bit codec evaluated in FP32, as the step evaluates it)
template <int Q, class S>
__device__ __forceinline__ void decode_pair_d(const S* __restrict__ src, int i, long long ps, size_t cell, int grp,
                                              const Args<float>& af, double& g, double& h) {
  if constexpr (IsS16<S>::value) {
    float gr, hr;
    ld_gh<Q, S, float>(src, i, ps, cell, gr, hr);
    g = static_cast<double>(gr * af.gref[grp]);
    h = static_cast<double>(hr * af.hscale[grp]);
  } else {
    ld_gh<Q, S, double>(src, i, ps, cell, g, h);
  }
}

// ---------------------------------------------------------------------------
// FP64 conservation sums of the deviations: per-block partials, then one
// fixed-order final pass; the host adds the reference totals N rho0 (mass)
// and N rho0 (D + delta) T0 / 2 (energy)
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 1024;
constexpr int kRedVals = 5;  // mass, momentum[3], energy

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int LAT, class S>
__global__ void __launch_bounds__(kRedThreads) k_conserve_partial(const S* __restrict__ src, long long N,
                                                                   const Args<double> a, const Args<float> af,
                                                                   double* __restrict__ partial) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  const long long ps = a.ps;
  double acc[kRedVals] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < N;
       cell += (long long)gridDim.x * blockDim.x) {
    static_for<Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      double gi, hi;
      decode_pair_d<Q, S>(src, i, ps, cell, L::grp(i), af, gi, hi);
      acc[0] += gi;
      if constexpr (L::cx(i) != 0) acc[1] += (a.r * L::cx(i)) * gi;
      if constexpr (L::cy(i) != 0) acc[2] += (a.r * L::cy(i)) * gi;
      if constexpr (L::cz(i) != 0) acc[3] += (a.r * L::cz(i)) * gi;
      acc[4] += a.half_r2 * L::c2(i) * gi + hi;
    });
  }
  __shared__ double sh[kRedThreads / 32][kRedVals];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kRedVals; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kRedVals) {
    double s = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) s += sh[w][threadIdx.x];
    partial[blockIdx.x * kRedVals + threadIdx.x] = s;
  }
}


}  // namespace lbm
