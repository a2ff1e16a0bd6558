// The finite-difference step of Sec. III (Eq. (16)/(17), third-order upwind
// convection) on a 2D lattice, marched along y with the planes split over
// warps.
//
// k_step_fd (kernels.cuh) gives each cell a thread that reads its own 74
// values and about 360 stencil values from global memory, most of them
// served by L2 (the y-neighbours lie a row pitch away, in rows other blocks
// load).  Here a block covers 32 columns of a band of rows with P warps and
// walks the band one row at a time.  The (c, -c) pairs of the lattice are
// dealt to the warps (pair p to warp p mod P; the rest velocity to warp
// P - 1); each warp streams the rows of its own planes through its own ring
// of R = 5 + L rows in shared memory (the 32 columns and 2 halo columns per
// side), so a value leaves global memory once per block, and every stencil
// value is a shared-memory read.  While a warp works on row y, the 4-byte
// cp.async copies of rows y + 3 .. y + 2 + L are in flight.  Per row:
//   1. each warp forms its pairs' partial moment sums; one block barrier;
//      every warp adds the P partial sums in warp order, so all warps hold
//      bitwise the same moments and equilibrium coefficients;
//   2. for each of its pairs, the equilibrium of c and -c (shared even part),
//      the upwind differences from its ring (rows y - 2 .. y + 2, columns
//      x - 2 .. x + 2), the relaxation and the store.
// Every warp runs one instruction stream: a pair's velocity, group and
// planes are per-thread values fixed at the kernel's start.
//
// A ring row holds the columns x0 - 2 .. x0 + 33 after the x rule (wrapped,
// or clamped at zero-gradient ends), and the ring row of row r holds grid
// row r after the y rule, so the stencil needs no boundary cases.  The
// arithmetic per value is that of k_step_fd; the moments are summed in
// another order (per warp, then over the warps), so the two kernels agree to
// rounding, not bitwise.
#pragma once

#include "launch_impl.cuh"

// warps per block (pairs per warp = 18 / P), rows in flight per warp, and
// the resident blocks per SM the register allocation aims at
#ifndef LBM_FD_MARCH_P
#define LBM_FD_MARCH_P 6
#endif
#ifndef LBM_FD_MARCH_L
#define LBM_FD_MARCH_L 1
#endif
#ifndef LBM_FD_MARCH_MINB
#define LBM_FD_MARCH_MINB 1
#endif

namespace lbm {

// the (c, -c) pairs of the library order (velocities 2p + 1, 2p + 2), each
// oriented so that its member c has c_y > 0, or c_y = 0 and c_x > 0
struct FdPair {
  int vc, vm;  // library indices of c and -c
  int cx, cy, c2, grp;
};

template <int LAT>
__host__ __device__ constexpr FdPair fd_pair(int p) {
  using L = Lat<LAT>;
  const int v = 2 * p + 1;
  const bool first = L::cy(v) > 0 || (L::cy(v) == 0 && L::cx(v) > 0);
  const int vc = first ? v : v + 1;
  return FdPair{vc, first ? v + 1 : v, L::cx(vc), L::cy(vc), L::c2(vc), L::grp(vc)};
}

// warp layout and ring geometry (in stored words: one value for FP64/FP32
// storage, one (g, h) pair for 16-bit storage)
template <int LAT, class S, int P, int L>
struct FdMarch {
  static constexpr bool SCALED = IsS16<S>::value;
  using Wd = typename std::conditional<SCALED, unsigned, S>::type;
  static constexpr int NPAIR = (Lat<LAT>::Q - 1) / 2;
  static constexpr int KP = NPAIR / P;         // pairs per warp
  static constexpr int PV = SCALED ? 1 : 2;    // stored words per velocity and cell
  static constexpr int PW = (2 * KP + 1) * PV; // ring planes of a warp: its pairs, then the rest velocity
  static constexpr int R = 5 + L;              // ring rows
  static constexpr int RW = 36;                // words of a ring row: 32 columns + 2 halo columns per side
  static constexpr int warp_words = R * PW * RW;
  static constexpr size_t ring_bytes = (size_t)P * warp_words * sizeof(Wd);
  // partial sums [row parity][5][P][32] in the compute type, after the rings
  template <class C>
  static constexpr size_t smem() {
    return (ring_bytes + 15) / 16 * 16 + 2 * 5 * P * 32 * sizeof(C);
  }
  static_assert(NPAIR % P == 0, "the pairs divide evenly over the warps");
};

template <int LAT, class S, class C, int P, int L, bool IDX32>
__global__ void __launch_bounds__(32 * P, LBM_FD_MARCH_MINB) k_step_fd_march(const S* __restrict__ src, S* __restrict__ dst,
                                                          const Args<C> a, C lamr, int nbands) {
  using Lt = Lat<LAT>;
  using M = FdMarch<LAT, S, P, L>;
  using Wd = typename M::Wd;
  static_assert(Lt::D == 2, "the marched step is written for 2D lattices");
  constexpr int Q = Lt::Q;
  constexpr int KP = M::KP, PV = M::PV, PW = M::PW, R = M::R, RW = M::RW;
  constexpr bool SCALED = M::SCALED;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  Wd* ring = reinterpret_cast<Wd*>(smem_raw) + w * M::warp_words;
  C* part = reinterpret_cast<C*>(smem_raw + (M::ring_bytes + 15) / 16 * 16);  // [2][5][P][32]

  const int nx = a.n[0], ny = a.n[1];
  const int x0 = blockIdx.x * 32;
  const int x = x0 + lane;
  const bool active = x < nx;
  const int yb = (int)((long long)ny * blockIdx.y / nbands);
  const int ye = (int)((long long)ny * (blockIdx.y + 1) / nbands);
  const long long ps = a.ps;
  const bool px = a.bc[0] == kPeriodic, py = a.bc[1] == kPeriodic;
  auto xmap = [&](int v) {
    if (px) {
      v %= nx;
      return v < 0 ? v + nx : v;
    }
    return v < 0 ? 0 : (v > nx - 1 ? nx - 1 : v);
  };
  auto ymap = [&](int v) {
    if (py) {
      v %= ny;
      return v < 0 ? v + ny : v;
    }
    return v < 0 ? 0 : (v > ny - 1 ? ny - 1 : v);
  };
  // source columns of this lane: its body column and (lanes 0..3) one halo
  // column, x0 - 2, x0 - 1, x0 + 32, x0 + 33; the halo's ring column
  const int sx_body = xmap(x);
  const int sx_halo = xmap(lane < 2 ? x0 - 2 + lane : x0 + 30 + lane);
  const int cx_halo = lane < 2 ? lane : 32 + lane;

  // this warp's pairs: velocity, group constants and library indices
  int pcx[KP], pcy[KP], plc[KP], plm[KP];
  C fcx[KP], fcy[KP], fc2[KP], x2[KP], wgt[KP], pref[KP], gref[KP], igref[KP], hsc[KP], ihsc[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const int p = w + P * k;
    FdPair q{};
    static_for<M::NPAIR>([&](auto I) {
      if (p == decltype(I)::value) q = fd_pair<LAT>(decltype(I)::value);
    });
    pcx[k] = q.cx;
    pcy[k] = q.cy;
    fcx[k] = C(q.cx);
    fcy[k] = C(q.cy);
    fc2[k] = C(q.c2);
    plc[k] = q.vc;
    plm[k] = q.vm;
    C gx2 = C(0), gw = C(0), gp = C(0), gr = C(0), ig = C(0), hs = C(0), ih = C(0);
    static_for<10>([&](auto G) {
      constexpr int g = decltype(G)::value;
      if (q.grp == g) {
        gx2 = a.x2g[g];
        gw = a.wg[g];
        gp = a.pref[g];
        gr = a.gref[g];
        ig = a.inv_gref[g];
        hs = a.hscale[g];
        ih = a.inv_hscale[g];
      }
    });
    x2[k] = gx2;
    wgt[k] = gw;
    pref[k] = gp;
    gref[k] = gr;
    igref[k] = ig;
    hsc[k] = hs;
    ihsc[k] = ih;
  }
  const bool has_rest = (w == P - 1);

  // copy grid row ymap(r) of every plane of this warp into its ring slot:
  // ring plane (2k + m) PV + q holds stored part q (g, h; or the pair) of
  // member m (0: c, 1: -c) of the warp's pair k; the rest velocity follows
  auto load_row = [&](int r) {
    const int s = (r - (yb - 2)) % R;
    const long long rowoff = (long long)ymap(r) * nx;
    Wd* dst_row = ring + s * PW * RW;
    auto cp = [&](int j, long long plane) {
      const Wd* srow = reinterpret_cast<const Wd*>(src) + plane * ps + rowoff;
      const unsigned d0 = (unsigned)__cvta_generic_to_shared(dst_row + j * RW + 2 + lane);
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d0), "l"(srow + sx_body),
                   "n"((int)sizeof(Wd))
                   : "memory");
      if (lane < 4) {
        const unsigned d1 = (unsigned)__cvta_generic_to_shared(dst_row + j * RW + cx_halo);
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d1), "l"(srow + sx_halo),
                     "n"((int)sizeof(Wd))
                     : "memory");
      }
    };
#pragma unroll
    for (int k = 0; k < KP; ++k) {
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int v = m ? plm[k] : plc[k];
#pragma unroll
        for (int q = 0; q < PV; ++q) cp((2 * k + m) * PV + q, SCALED ? (long long)v : (long long)q * Q + v);
      }
    }
    if (has_rest) {
#pragma unroll
      for (int q = 0; q < PV; ++q) cp(2 * KP * PV + q, SCALED ? 0LL : (long long)q * Q);
    }
  };
  auto commit = [] { asm volatile("cp.async.commit_group;\n" ::: "memory"); };

  // prologue: rows yb - 2 .. yb + 2 + L, one commit group per row (rows past
  // ye + 1 are not needed: empty groups keep the count)
  for (int r = yb - 2; r <= yb + 2 + L; ++r) {
    if (r <= ye + 1) load_row(r);
    commit();
  }

  const int col = 2 + lane;
  for (int y = yb; y < ye; ++y) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(L) : "memory");
    __syncwarp();
    auto rowp = [&](int r) -> const Wd* { return ring + ((r - (yb - 2)) % R) * PW * RW; };
    const Wd* rm2 = rowp(y - 2);
    const Wd* rm1 = rowp(y - 1);
    const Wd* r0 = rowp(y);
    const Wd* rp1 = rowp(y + 1);
    const Wd* rp2 = rowp(y + 2);
    // (g, h) of velocity slot j (2k + m, or 2 KP for the rest) at a ring row and column
    auto val = [&](const Wd* row, int j, int c, C& g, C& h) {
      if constexpr (SCALED) {
        float lo, hi;
        unpack16<S>(row[j * RW + c], lo, hi);
        g = static_cast<C>(lo);
        h = static_cast<C>(hi);
      } else {
        g = static_cast<C>(row[(2 * j) * RW + c]);
        h = static_cast<C>(row[(2 * j + 1) * RW + c]);
      }
    };
    // own values and this warp's partial moment sums (16-bit storage: the
    // group scales fold into the coefficients, as in moments_raw)
    C gc[KP], hc[KP], gm[KP], hm[KP], g0 = C(0), h0 = C(0);
    C sm = C(0), sjx = C(0), sjy = C(0), sk2 = C(0), sH = C(0);
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      val(r0, 2 * k, col, gc[k], hc[k]);
      val(r0, 2 * k + 1, col, gm[k], hm[k]);
      const C sp = gc[k] + gm[k], df = gc[k] - gm[k], hp = hc[k] + hm[k];
      if constexpr (SCALED) {
        sm = fma(gref[k], sp, sm);
        sjx = fma(fcx[k] * gref[k], df, sjx);
        sjy = fma(fcy[k] * gref[k], df, sjy);
        sk2 = fma(fc2[k] * gref[k], sp, sk2);
        sH = fma(hsc[k], hp, sH);
      } else {
        sm += sp;
        sjx = fma(fcx[k], df, sjx);
        sjy = fma(fcy[k], df, sjy);
        sk2 = fma(fc2[k], sp, sk2);
        sH += hp;
      }
    }
    if (has_rest) {
      val(r0, 2 * KP, col, g0, h0);
      if constexpr (SCALED) {
        sm = fma(a.gref[0], g0, sm);
        sH = fma(a.hscale[0], h0, sH);
      } else {
        sm += g0;
        sH += h0;
      }
    }
    C* pb = part + (y & 1) * 5 * P * 32;
    pb[(0 * P + w) * 32 + lane] = sm;
    pb[(1 * P + w) * 32 + lane] = sjx;
    pb[(2 * P + w) * 32 + lane] = sjy;
    pb[(3 * P + w) * 32 + lane] = C(0);
    pb[(4 * P + w) * 32 + lane] = fma(a.half_r2, sk2, sH);
    __syncthreads();
    C acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      C t = pb[(q * P) * 32 + lane];
#pragma unroll
      for (int v = 1; v < P; ++v) t += pb[(q * P + v) * 32 + lane];
      acc[q] = t;
    }
    C drho, u[3], dT;
    moments_finish<LAT, C>(acc, a, drho, u, dT);
    if (w == 0 && active && !(isfinite(drho) && isfinite(dT))) atomicOr(a.flag, 1u);
    EqCoef<LAT, C> kc;
    eq_coeffs<LAT, C>(drho, u, dT, a, kc);
    const C hA = a.omega_g * a.half_delta * kc.T;
    const C om1 = C(1) - a.omega_g;
    const C hbs = a.omega_g * a.half_delta * kc.dT;
    const unsigned cell = (unsigned)x + (unsigned)nx * (unsigned)y;
    auto store = [&](int v, C gn, C hn) {
      if constexpr (SCALED) {
        unsigned* dp = reinterpret_cast<unsigned*>(dst);
        const unsigned pv = pack16<S>(static_cast<float>(gn), static_cast<float>(hn));
        if constexpr (IDX32) dp[(unsigned)v * (unsigned)ps + cell] = pv;
        else dp[(size_t)v * ps + cell] = pv;
      } else {
        if constexpr (IDX32) {
          dst[(unsigned)v * (unsigned)ps + cell] = static_cast<S>(gn);
          dst[(unsigned)(Q + v) * (unsigned)ps + cell] = static_cast<S>(hn);
        } else {
          dst[(size_t)v * ps + cell] = static_cast<S>(gn);
          dst[(size_t)(Q + v) * ps + cell] = static_cast<S>(hn);
        }
      }
    };
    // the upwind difference of k_step_fd from the values at the upwind-2,
    // upwind-1 and downwind-1 positions (sg: the sign of the component)
    auto upwind = [&](C sg, C gm2, C hm2, C gm1, C hm1, C gp1, C hp1, C og, C oh, C& dg, C& dh) {
      dg = sg * (gm2 - C(6) * gm1 + C(3) * og + C(2) * gp1) * C(1.0 / 6.0);
      dh = sg * (hm2 - C(6) * hm1 + C(3) * oh + C(2) * hp1) * C(1.0 / 6.0);
    };
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      // equilibrium of the pair (eq_emit's forms with this pair's group)
      const C Pg = fma(x2[k], fma(x2[k], kc.pc, kc.pb), kc.pa);
      const C W = wgt[k] * kc.rho;
      const C c0 = wgt[k] * fma(kc.drho, C(1) + Pg, a.rho0 * (Pg - pref[k]));
      const C c1 = W * fma(kc.be1, x2[k], kc.be0);
      const C c2 = W * fma(kc.ga1, x2[k], kc.ga0);
      const C c3 = W * C(1.0 / 6.0);
      const C c4 = W * C(1.0 / 24.0);
      C s = fma(fcx[k], kc.ur[0], C(0));
      s = fma(fcy[k], kc.ur[1], s);
      const C s2 = s * s;
      const C e = fma(s2, fma(s2, c4, c2), c0);
      const C o = s * fma(s2, c3, c1);
      // convection of c and of -c, x part then y part
      C cgc = C(0), chc = C(0), cgm = C(0), chm = C(0);
      if (pcx[k] != 0) {
        const int sx = pcx[k] > 0 ? 1 : -1;
        C a2, b2, a1, b1, ap, bp, dg, dh;
        val(r0, 2 * k, col - 2 * sx, a2, b2);
        val(r0, 2 * k, col - sx, a1, b1);
        val(r0, 2 * k, col + sx, ap, bp);
        upwind(C(sx), a2, b2, a1, b1, ap, bp, gc[k], hc[k], dg, dh);
        cgc = fma(fcx[k], dg, cgc);
        chc = fma(fcx[k], dh, chc);
        val(r0, 2 * k + 1, col + 2 * sx, a2, b2);
        val(r0, 2 * k + 1, col + sx, a1, b1);
        val(r0, 2 * k + 1, col - sx, ap, bp);
        upwind(C(-sx), a2, b2, a1, b1, ap, bp, gm[k], hm[k], dg, dh);
        cgm = fma(-fcx[k], dg, cgm);
        chm = fma(-fcx[k], dh, chm);
      }
      if (pcy[k] != 0) {  // c_y > 0 for the member c
        C a2, b2, a1, b1, ap, bp, dg, dh;
        val(rm2, 2 * k, col, a2, b2);
        val(rm1, 2 * k, col, a1, b1);
        val(rp1, 2 * k, col, ap, bp);
        upwind(C(1), a2, b2, a1, b1, ap, bp, gc[k], hc[k], dg, dh);
        cgc = fma(fcy[k], dg, cgc);
        chc = fma(fcy[k], dh, chc);
        val(rp2, 2 * k + 1, col, a2, b2);
        val(rp1, 2 * k + 1, col, a1, b1);
        val(rm1, 2 * k + 1, col, ap, bp);
        upwind(C(-1), a2, b2, a1, b1, ap, bp, gm[k], hm[k], dg, dh);
        cgm = fma(-fcy[k], dg, cgm);
        chm = fma(-fcy[k], dh, chm);
      }
      // relax (relax_store_k's forms) and subtract the convection
      auto relax = [&](C dF, C gv, C hv, C cg, C ch, int v) {
        C gn, hn;
        if constexpr (SCALED) {
          gn = fma(a.omega_f, fma(dF, igref[k], -gv), gv);
          hn = fma(hA * ihsc[k], dF, fma(om1, hv, hbs * gref[k] * ihsc[k]));
        } else {
          gn = fma(a.omega_f, dF - gv, gv);
          hn = fma(hA, dF, fma(om1, hv, hbs * gref[k]));
        }
        gn -= lamr * cg;
        hn -= lamr * ch;
        if (active) store(v, gn, hn);
      };
      relax(e + o, gc[k], hc[k], cgc, chc, plc[k]);
      relax(e - o, gm[k], hm[k], cgm, chm, plm[k]);
    }
    if (has_rest) {
      // group 0 has x2 = 0: the equilibrium deviation is its c0
      const C Pg = kc.pa;
      const C c0 = a.wg[0] * fma(kc.drho, C(1) + Pg, a.rho0 * (Pg - a.pref[0]));
      C gn, hn;
      if constexpr (SCALED) {
        gn = fma(a.omega_f, fma(c0, a.inv_gref[0], -g0), g0);
        hn = fma(hA * a.inv_hscale[0], c0, fma(om1, h0, hbs * a.gref[0] * a.inv_hscale[0]));
      } else {
        gn = fma(a.omega_f, c0 - g0, g0);
        hn = fma(hA, c0, fma(om1, h0, hbs * a.gref[0]));
      }
      if (active) store(0, gn, hn);
    }
    // every lane is done with the ring row of y - 2: copy row y + 3 + L there
    __syncwarp();
    if (y + 3 + L <= ye + 1) load_row(y + 3 + L);
    commit();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// launch
// ---------------------------------------------------------------------------
inline bool fd_march_fits(const Instance* inst) { return inst->D == 2; }

// Bands per strip: the grid of strips x bands should fill whole waves of
// resident blocks, and each band re-reads 4 halo rows, so the choice
// maximises (blocks / slots of the waves) x rows / (rows + 4).
inline int fd_march_bands(int nstrips, int ny, int resident) {
  int best = 1;
  double best_eff = 0.0;
  const int max_nb = ny < 4096 ? ny : 4096;
  for (int nb = 1; nb <= max_nb; ++nb) {
    const long long blocks = (long long)nstrips * nb;
    const long long waves = (blocks + resident - 1) / resident;
    const double rows = (double)ny / nb;
    const double eff = (double)blocks / (double)(waves * resident) * rows / (rows + 4.0);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = nb;
    }
  }
  return best;
}

template <int LAT, class S, class C, int P, int L, bool IDX32>
cudaError_t launch_fd_march_v(const Instance* inst, const void* src, void* dst, double lam) {
  using M = FdMarch<LAT, S, P, L>;
  constexpr size_t smem = M::template smem<C>();
  auto kern = k_step_fd_march<LAT, S, C, P, L, IDX32>;
  // per device (bit d): the shared-memory opt-in and the resident blocks
  static std::atomic<unsigned long long> configured{0};
  static std::atomic<int> resident_of[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64) return cudaErrorInvalidDevice;
  if (!(configured.load(std::memory_order_acquire) & (1ull << dev))) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * P, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    resident_of[dev].store(per_sm * sms, std::memory_order_relaxed);
    configured.fetch_or(1ull << dev, std::memory_order_release);
  }
  const int nstrips = (inst->n[0] + 31) / 32;
  const int nb = fd_march_bands(nstrips, inst->n[1], resident_of[dev].load(std::memory_order_relaxed));
  const Args<C>& a = args_of<C>(inst);
  kern<<<dim3((unsigned)nstrips, (unsigned)nb), 32 * P, smem, inst->stream>>>(
      static_cast<const S*>(src), static_cast<S*>(dst), a, static_cast<C>(lam * inst->table.r), nb);
  return cudaGetLastError();
}

template <int LAT, class S, class C>
cudaError_t launch_fd_march_t(const Instance* inst, const void* src, void* dst, double lam) {
  const long long planes = IsS16<S>::value ? Lat<LAT>::Q : 2LL * Lat<LAT>::Q;
  if (planes * inst->ps < (1LL << 32))
    return launch_fd_march_v<LAT, S, C, LBM_FD_MARCH_P, LBM_FD_MARCH_L, true>(inst, src, dst, lam);
  return launch_fd_march_v<LAT, S, C, LBM_FD_MARCH_P, LBM_FD_MARCH_L, false>(inst, src, dst, lam);
}

// the finite-difference step: the per-cell kernel k_step_fd, or the marched
// kernel on 2D grids when the instance asked for it
template <int LAT, class S, class C>
cudaError_t launch_step_fd_any(const Instance* inst, const void* src, void* dst, double lam) {
  if constexpr (Lat<LAT>::D == 2) {
    if (inst->fd_kernel == LBM_FD_MARCH && fd_march_fits(inst)) return launch_fd_march_t<LAT, S, C>(inst, src, dst, lam);
  }
  return launch_step_fd_t<LAT, S, C>(inst, src, dst, lam);
}

}  // namespace lbm
