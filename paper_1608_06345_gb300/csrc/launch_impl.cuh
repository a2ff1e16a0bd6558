// Launcher templates: pick the step shape, set up and launch the kernels of
// one (lattice, storage type, compute type).
#pragma once

#include <atomic>

#include "runtime.h"

namespace lbm {

template <class C>
const Args<C>& args_of(const Instance* inst) {
  if constexpr (std::is_same<C, double>::value) return inst->ad;
  else return inst->af;
}

// dynamic shared memory of a step shape: none (STAGE 0, 6), h only (STAGE 3),
// g and h (STAGE 1, 2)
template <int LAT, class S, int STAGE, int BX>
constexpr size_t step_smem() {
  if constexpr (STAGE == 9) return sizeof(unsigned) * (Lat<LAT>::Q - (Lat<LAT>::Q + 1) / 2) * BX;
  return (STAGE == 0 || STAGE == 6) ? 0 : (STAGE == 3 ? 1 : 2) * sizeof(S) * Lat<LAT>::Q * BX;
}

// the dynamic shared-memory opt-in is a per-device function attribute: set
// it once per device (bit d of the mask) for each kernel instance; the mask
// is atomic because host threads may launch concurrently (setting the
// attribute twice is harmless)
template <int LAT, class S, class C, int STAGE, int BX, int MINB, bool IDX32, int ROWS>
cudaError_t step_smem_opt_in(size_t smem) {
  static std::atomic<unsigned long long> configured{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !(configured.load(std::memory_order_acquire) & (1ull << dev))) {
    e = cudaFuncSetAttribute(k_step<LAT, S, C, STAGE, BX, MINB, IDX32, ROWS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dev < 64) configured.fetch_or(1ull << dev, std::memory_order_release);
  }
  return cudaSuccess;
}

// rows of a 3D grid that lie within 3 cells of a y or z face
inline long long boundary_rows(int ny, int nz) { return (long long)ny * nz - (long long)(ny - 6) * (nz - 6); }

template <int LAT, class S, class C, int STAGE, int BX, int MINB = 1, bool IDX32 = false>
cudaError_t launch_step_v(const Instance* inst, const void* src, void* dst, const Args<C>& a,
                          bool configure_only = false) {
  constexpr size_t smem = step_smem<LAT, S, STAGE, BX>();
  const unsigned gx = (unsigned)((inst->n[0] + BX - 1) / BX);
  // a 3D grid with interior rows whose byte offsets fit 32 bits (the ROW
  // path): with FP32 storage and 32-bit element indices one launch whose
  // every block takes the ROW path's code with block-uniform row shift
  // tables; otherwise an interior and a boundary launch (measured: the
  // uniform launch is the faster for FP32 storage, the split for 16-bit)
  constexpr long long E = IsS16<S>::value ? 2 * (long long)sizeof(S) : (long long)sizeof(S);
  constexpr bool UNIFORM = Lat<LAT>::D == 3 && IDX32 && sizeof(S) == 4 && !IsS16<S>::value;
  const int ny = inst->n[1], nz = inst->n[2];
  const bool split = Lat<LAT>::D == 3 && ny >= 7 && nz >= 7 && inst->N * E < (1LL << 32) &&
                     boundary_rows(ny, nz) <= 65535;
  // (the choice is made at compile time where it can be, so that no kernel
  // instance is built that a launch never reaches)
  if constexpr (smem != 0) {
    cudaError_t e;
    if constexpr (UNIFORM) {
      e = split ? step_smem_opt_in<LAT, S, C, STAGE, BX, MINB, IDX32, kRowsUniform>(smem)
                : step_smem_opt_in<LAT, S, C, STAGE, BX, MINB, IDX32, kRowsAll>(smem);
    } else {
      e = split ? step_smem_opt_in<LAT, S, C, STAGE, BX, MINB, IDX32, kRowsInterior>(smem)
                : step_smem_opt_in<LAT, S, C, STAGE, BX, MINB, IDX32, kRowsAll>(smem);
      if (e == cudaSuccess && split) e = step_smem_opt_in<LAT, S, C, STAGE, BX, MINB, IDX32, kRowsBoundary>(smem);
    }
    if (e != cudaSuccess) return e;
  }
  if (configure_only) return cudaSuccess;
  const S* s = static_cast<const S*>(src);
  S* d = static_cast<S*>(dst);
  if constexpr (UNIFORM) {
    if (split) {
      k_step<LAT, S, C, STAGE, BX, MINB, IDX32, kRowsUniform>
          <<<dim3(gx, (unsigned)ny, (unsigned)nz), BX, smem, inst->stream>>>(s, d, a);
      return cudaGetLastError();
    }
  } else if constexpr (Lat<LAT>::D == 3) {
    if (split) {
      k_step<LAT, S, C, STAGE, BX, MINB, IDX32, kRowsInterior>
          <<<dim3(gx, (unsigned)(ny - 6), (unsigned)(nz - 6)), BX, smem, inst->stream>>>(s, d, a);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      k_step<LAT, S, C, STAGE, BX, MINB, IDX32, kRowsBoundary>
          <<<dim3(gx, (unsigned)boundary_rows(ny, nz), 1), BX, smem, inst->stream>>>(s, d, a);
      return cudaGetLastError();
    }
  }
  k_step<LAT, S, C, STAGE, BX, MINB, IDX32, kRowsAll>
      <<<dim3(gx, (unsigned)ny, (unsigned)nz), BX, smem, inst->stream>>>(s, d, a);
  return cudaGetLastError();
}

// Buffers whose element indices (2Q ps; Q ps pairs for 16-bit storage) stay
// below 2^32 index in unsigned 32-bit arithmetic, which takes fewer integer
// instructions per load and store (4096^2 D2Q37 and 256^3 D3Q107 both do)
template <int LAT, class S, class C, int STAGE, int BX, int MINB = 1>
cudaError_t launch_step_t(const Instance* inst, const void* src, void* dst, const Args<C>& a,
                          bool configure_only = false) {
  const long long planes = IsS16<S>::value ? Lat<LAT>::Q : 2LL * Lat<LAT>::Q;
  if (planes * inst->ps < (1LL << 32))
    return launch_step_v<LAT, S, C, STAGE, BX, MINB, true>(inst, src, dst, a, configure_only);
  return launch_step_v<LAT, S, C, STAGE, BX, MINB, false>(inst, src, dst, a, configure_only);
}

// the velocity-split step: 32 cells per block, P warps (static shared memory only)
template <int LAT, class S, class C, int P, int MINB, bool SHARE = false>
cudaError_t launch_step_split(const Instance* inst, const void* src, void* dst, const Args<C>& a,
                              bool configure_only = false) {
  if (configure_only) return cudaSuccess;
  const dim3 grid((unsigned)((inst->n[0] + 31) / 32), (unsigned)inst->n[1], (unsigned)inst->n[2]);
  k_step_split<LAT, S, C, P, MINB, SHARE><<<grid, dim3(32, P), 0, inst->stream>>>(static_cast<const S*>(src),
                                                                           static_cast<S*>(dst), a);
  return cudaGetLastError();
}

// the mirror-pair step (stage 8): BX threads, BX / 2 cells per block; HS
// stages h in shared memory (FP32/FP64 storage)
template <int LAT, class S, class C, int BX, int MINB, bool HS, bool IDX32>
cudaError_t launch_step_mirror_v(const Instance* inst, const void* src, void* dst, const Args<C>& a,
                                 bool configure_only) {
  constexpr size_t smem = HS ? sizeof(S) * ((Lat<LAT>::Q - 1) / 2) * BX : 0;
  if constexpr (smem > 48 * 1024) {
    // per-device shared-memory opt-in, as in launch_step_v
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !(configured.load(std::memory_order_acquire) & (1ull << dev))) {
      e = cudaFuncSetAttribute(k_step_mirror<LAT, S, C, BX, MINB, IDX32, HS>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      if (dev < 64) configured.fetch_or(1ull << dev, std::memory_order_release);
    }
  }
  if (configure_only) return cudaSuccess;
  const dim3 grid((unsigned)((inst->n[0] + BX / 2 - 1) / (BX / 2)), (unsigned)inst->n[1], (unsigned)inst->n[2]);
  k_step_mirror<LAT, S, C, BX, MINB, IDX32, HS><<<grid, BX, smem, inst->stream>>>(static_cast<const S*>(src),
                                                                                 static_cast<S*>(dst), a);
  return cudaGetLastError();
}

template <int LAT, class S, class C, int BX, int MINB, bool HS>
cudaError_t launch_step_mirror(const Instance* inst, const void* src, void* dst, const Args<C>& a,
                               bool configure_only = false) {
  const long long planes = IsS16<S>::value ? Lat<LAT>::Q : 2LL * Lat<LAT>::Q;
  if (planes * inst->ps < (1LL << 32))
    return launch_step_mirror_v<LAT, S, C, BX, MINB, HS, true>(inst, src, dst, a, configure_only);
  return launch_step_mirror_v<LAT, S, C, BX, MINB, HS, false>(inst, src, dst, a, configure_only);
}

// Candidate shapes of the step per (lattice, storage), tried by the
// autotuner; index 0 is the default.  (stage, cells per block, minimum
// resident blocks per SM requested from the compiler, which caps registers):
//   D2Q37 FP32:        (0,128,4) (0,256,2) (0,64,8) (0,128,1)
//   D2Q37 16-bit:      (6,128,8) (6,128,7) (6,128,6) (6,256,3) (0,128,4) (0,64,8)
//   D2Q37 FP64:        (0,128,1) (0,256,1) (0,64,1)  (4,32,4)  (7,32,4)
//   D3Q107 FP32:       (3,64,6)  (3,64,1)  (1,64,1)  (4,32,6)  (8,32,8)  (8,64,4)  (3,128,3)
//   D3Q107 FP64:       (1,64,1)  (4,32,3)  (4,32,2)  (7,32,3)
//   D3Q107 16-bit:     (6,64,6)  (9,256,2) (2,64,1)  (4,32,6)  (8,32,10) (8,32,12) (6,128,3)
// Stage 4 is the velocity-split step: 4 warps per block of 32 cells; stage 7
// the same with the per-cell coefficients formed once by warp 0 and shared.
// Stage 8 is the mirror-pair step: two lanes per cell (c and -c of every
// pair), h staged in shared memory for FP32.  Stage 9 holds half the 16-bit
// pairs packed in registers and stages the other half in shared memory.  The moments of stages 4, 7
// and 8 are summed in another order, so their results differ from the
// other shapes' by rounding; the defaults (index 0) are the shapes the
// batched pool uses, whose results are bitwise those of a lone instance.
template <int LAT, class S>
struct StepShapes {
  static constexpr int count =
      (LAT == 0) ? (sizeof(S) == 8 ? 5 : (sizeof(S) == 2 ? 6 : 4)) : (sizeof(S) == 8 ? 4 : 7);
  static void get(int k, int* stage, int* bx, int* minb) {
    static const int s2[4][3] = {{0, 128, 4}, {0, 256, 2}, {0, 64, 8}, {0, 128, 1}};
    static const int s2h[6][3] = {{6, 128, 8}, {6, 128, 7}, {6, 128, 6}, {6, 256, 3}, {0, 128, 4}, {0, 64, 8}};
    static const int s2d[5][3] = {{0, 128, 1}, {0, 256, 1}, {0, 64, 1}, {4, 32, 4}, {7, 32, 4}};
    static const int s3f[7][3] = {{3, 64, 6}, {3, 64, 1}, {1, 64, 1}, {4, 32, 6}, {8, 32, 8}, {8, 64, 4}, {3, 128, 3}};
    static const int s3d[4][3] = {{1, 64, 1}, {4, 32, 3}, {4, 32, 2}, {7, 32, 3}};
    static const int s3h[7][3] = {{6, 64, 6}, {9, 256, 2}, {2, 64, 1}, {4, 32, 6}, {8, 32, 10}, {8, 32, 12}, {6, 128, 3}};
    const int(*t)[3] = (LAT == 0) ? (sizeof(S) == 8 ? s2d : (sizeof(S) == 2 ? s2h : s2))
                                  : (sizeof(S) == 4 ? s3f : (sizeof(S) == 8 ? s3d : s3h));
    *stage = t[k][0];
    *bx = t[k][1];
    *minb = t[k][2];
  }
};

template <int LAT, class S>
int shape_count_t() { return StepShapes<LAT, S>::count; }

template <int LAT, class S>
void shape_get_t(int k, int* stage, int* bx) {
  int minb = 1;
  StepShapes<LAT, S>::get(k, stage, bx, &minb);
}

template <int LAT, class S, class C>
cudaError_t launch_step_shape(const Instance* inst, const void* src, void* dst, bool configure_only = false) {
  const Args<C>& a = args_of<C>(inst);
  const int k = inst->shape.index;
  if constexpr (LAT == 0 && sizeof(S) == 8) {
    switch (k) {
      case 1: return launch_step_t<LAT, S, C, 0, 256>(inst, src, dst, a, configure_only);
      case 2: return launch_step_t<LAT, S, C, 0, 64>(inst, src, dst, a, configure_only);
      case 3: return launch_step_split<LAT, S, C, 4, 4>(inst, src, dst, a, configure_only);
      case 4: return launch_step_split<LAT, S, C, 4, 4, true>(inst, src, dst, a, configure_only);
      default: return launch_step_t<LAT, S, C, 0, 128>(inst, src, dst, a, configure_only);
    }
  } else if constexpr (LAT == 0 && sizeof(S) == 2) {
    switch (k) {
      case 1: return launch_step_t<LAT, S, C, 6, 128, 7>(inst, src, dst, a, configure_only);
      case 2: return launch_step_t<LAT, S, C, 6, 128, 6>(inst, src, dst, a, configure_only);
      case 3: return launch_step_t<LAT, S, C, 6, 256, 3>(inst, src, dst, a, configure_only);
      case 4: return launch_step_t<LAT, S, C, 0, 128, 4>(inst, src, dst, a, configure_only);
      case 5: return launch_step_t<LAT, S, C, 0, 64, 8>(inst, src, dst, a, configure_only);
      default: return launch_step_t<LAT, S, C, 6, 128, 8>(inst, src, dst, a, configure_only);
    }
  } else if constexpr (LAT == 0) {
    switch (k) {
      case 1: return launch_step_t<LAT, S, C, 0, 256, 2>(inst, src, dst, a, configure_only);
      case 2: return launch_step_t<LAT, S, C, 0, 64, 8>(inst, src, dst, a, configure_only);
      case 3: return launch_step_t<LAT, S, C, 0, 128, 1>(inst, src, dst, a, configure_only);
      default: return launch_step_t<LAT, S, C, 0, 128, 4>(inst, src, dst, a, configure_only);
    }
  } else if constexpr (sizeof(S) == 4) {
    switch (k) {
      case 1: return launch_step_t<LAT, S, C, 3, 64>(inst, src, dst, a, configure_only);
      case 2: return launch_step_t<LAT, S, C, 1, 64>(inst, src, dst, a, configure_only);
      case 3: return launch_step_split<LAT, S, C, 4, 6>(inst, src, dst, a, configure_only);
      case 4: return launch_step_mirror<LAT, S, C, 64, 8, true>(inst, src, dst, a, configure_only);
      case 5: return launch_step_mirror<LAT, S, C, 128, 4, true>(inst, src, dst, a, configure_only);
      case 6: return launch_step_t<LAT, S, C, 3, 128, 3>(inst, src, dst, a, configure_only);
      default: return launch_step_t<LAT, S, C, 3, 64, 6>(inst, src, dst, a, configure_only);
    }
  } else if constexpr (sizeof(S) == 8) {
    switch (k) {
      case 1: return launch_step_split<LAT, S, C, 4, 3>(inst, src, dst, a, configure_only);
      case 2: return launch_step_split<LAT, S, C, 4, 2>(inst, src, dst, a, configure_only);
      case 3: return launch_step_split<LAT, S, C, 4, 3, true>(inst, src, dst, a, configure_only);
      default: return launch_step_t<LAT, S, C, 1, 64>(inst, src, dst, a, configure_only);
    }
  } else {
    switch (k) {
      case 1: return launch_step_t<LAT, S, C, 9, 256, 2>(inst, src, dst, a, configure_only);
      case 2: return launch_step_t<LAT, S, C, 2, 64>(inst, src, dst, a, configure_only);
      case 3: return launch_step_split<LAT, S, C, 4, 6>(inst, src, dst, a, configure_only);
      case 4: return launch_step_mirror<LAT, S, C, 64, 10, false>(inst, src, dst, a, configure_only);
      case 5: return launch_step_mirror<LAT, S, C, 64, 12, false>(inst, src, dst, a, configure_only);
      case 6: return launch_step_t<LAT, S, C, 6, 128, 3>(inst, src, dst, a, configure_only);
      default: return launch_step_t<LAT, S, C, 6, 64, 6>(inst, src, dst, a, configure_only);
    }
  }
}

// sets the shape's kernel attributes on the current device without
// launching (done before a graph capture)
template <int LAT, class S, class C>
cudaError_t configure_step_t(const Instance* inst) {
  return launch_step_shape<LAT, S, C>(inst, nullptr, nullptr, true);
}

template <int LAT, class S, class C>
cudaError_t launch_step_plain(const Instance* inst, const void* src, void* dst) {
  return launch_step_shape<LAT, S, C>(inst, src, dst, false);
}

// the finite-difference step (lam = dt/dx): 128 cells per block in 2D, 64 in 3D
template <int LAT, class S, class C>
cudaError_t launch_step_fd_t(const Instance* inst, const void* src, void* dst, double lam) {
  constexpr int BX = (LAT == 0) ? 128 : 64;
  const dim3 grid((unsigned)((inst->n[0] + BX - 1) / BX), (unsigned)inst->n[1], (unsigned)inst->n[2]);
  const Args<C>& a = args_of<C>(inst);
  k_step_fd<LAT, S, C, BX><<<grid, BX, 0, inst->stream>>>(static_cast<const S*>(src), static_cast<S*>(dst), a,
                                                          static_cast<C>(lam * inst->table.r));
  return cudaGetLastError();
}

// pool: the shape of the batched step per (lattice, storage)
template <int LAT, class S>
struct PoolShape {
  static constexpr int kStage = (LAT == 0) ? 0 : (sizeof(S) == 4 ? 3 : (sizeof(S) == 8 ? 1 : 2));
  static constexpr int kBX = (LAT == 0) ? 128 : 64;
};

template <int LAT, class S, class C>
cudaError_t launch_pool_step_t(const PoolLaunch& pl) {
  using PS = PoolShape<LAT, S>;
  auto kern = k_pool_step<LAT, S, C, PS::kStage, PS::kBX>;
  // the shared-memory opt-in was set by pool_grid_t at pool creation (outside
  // any stream capture)
  const size_t smem = step_smem<LAT, S, PS::kStage, PS::kBX>();
  kern<<<pl.grid, PS::kBX, smem, pl.stream>>>(static_cast<const PoolSlot<C>*>(pl.slots), pl.tiles, pl.ntiles);
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_pool_advance_t(const PoolLaunch& pl) {
  const int t = 128;
  k_pool_advance<C><<<(pl.nslots + t - 1) / t, t, 0, pl.stream>>>(static_cast<PoolSlot<C>*>(pl.slots), pl.nslots);
  return cudaGetLastError();
}

// persistent grid of the batched step: resident blocks per SM x SMs
template <int LAT, class S, class C>
int pool_grid_t() {
  using PS = PoolShape<LAT, S>;
  const size_t smem = step_smem<LAT, S, PS::kStage, PS::kBX>();
  auto kern = k_pool_step<LAT, S, C, PS::kStage, PS::kBX>;
  if (smem && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PS::kBX, smem) != cudaSuccess) return 0;
  return sms * (per_sm > 0 ? per_sm : 1);
}

template <int LAT, class S>
constexpr int pool_tile_cells() { return PoolShape<LAT, S>::kBX; }

inline unsigned blocks_for(long long N, int t) { return (unsigned)((N + t - 1) / t); }


template <int LAT, class S, class C>
cudaError_t launch_init_t(const Instance* inst, void* dst, const double* rho, const double* u, const double* T) {
  constexpr int kT = 128;
  if (inst->N == 0) return cudaSuccess;
  k_init<LAT, S, C><<<blocks_for(inst->N, kT), kT, 0, inst->stream>>>(static_cast<S*>(dst), rho, u, T, inst->N,
                                                                      args_of<C>(inst), inst->rho0, inst->T0);
  return cudaGetLastError();
}


template <int LAT, class S, class C>
cudaError_t launch_moments_t(const Instance* inst, const void* src, double* rho, double* u, double* T) {
  constexpr int kT = 128;
  if (inst->N == 0) return cudaSuccess;
  k_moments<LAT, S, C><<<blocks_for(inst->N, kT), kT, 0, inst->stream>>>(
      static_cast<const S*>(src), rho, u, T, inst->N, args_of<C>(inst), inst->rho0, inst->T0);
  return cudaGetLastError();
}


template <int LAT, class S>
cudaError_t launch_conserve_t(const Instance* inst, const void* src, double* partial, int nblocks) {
  k_conserve_partial<LAT, S><<<nblocks, kRedThreads, 0, inst->stream>>>(static_cast<const S*>(src), inst->N,
                                                                         inst->ad, inst->af, partial);
  return cudaGetLastError();
}


}  // namespace lbm
