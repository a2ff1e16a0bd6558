// Conservation totals without any device allocation (lbm_conserved_noalloc).
//
// Who needs it: callers that keep the populations in device memory owned by
// someone else and cannot call cudaMalloc at the point where they want the
// totals -- for example a serving pool that has reserved the whole device
// budget up front (a new allocation would fail, or stall the device while
// the allocator synchronises), or an application that restored a checkpoint
// into its own arena and has no library instance to borrow scratch from.
//
// The block partials of the reduction live in the file-scope array below
// instead of instance memory.  It has a fixed size of kNaMaxBlocks * 5 + 5
// doubles (about 160 KB); every GPU that loads the library holds it until
// the process exits.  One block covers kNaCellsPerBlock cells, so at most
// kNaMaxCells cells are accepted.  All calls share the array: calls that
// overlap on the GPU (different streams, or host threads) race on it.
#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "kernels.cuh"
#include "runtime.h"

namespace lbm {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaCellsPerThread = 16;
constexpr long long kNaCellsPerBlock = (long long)kNaThreads * kNaCellsPerThread;  // 4096
constexpr int kNaMaxBlocks = 4096;
constexpr long long kNaMaxCells = kNaCellsPerBlock * kNaMaxBlocks;               // 16,777,216
constexpr int kNaSlots = kNaMaxBlocks * kRedVals + kRedVals;                     // partials + totals

static __device__ __align__(256) double g_noalloc_scratch[kNaSlots];

// Per-device address of g_noalloc_scratch.  In host code the symbol name is
// a host-side stand-in, not a device address, so it is looked up once per
// device (with that device current) and only the looked-up pointer is
// passed to the kernels.
std::mutex g_addr_mutex;
double* g_addr[64] = {};

int scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(LBM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return set_error(LBM_EINVAL, "device index above 63");
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return set_error(LBM_ECUDA, std::string("cudaGetSymbolAddress of the scratch array: ") + cudaGetErrorString(e));
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return LBM_OK;
}

// Partial sums of the deviations over one contiguous chunk of cells per block.
template <int LAT, class S>
__global__ void __launch_bounds__(kNaThreads) k_conserve_chunk(const S* __restrict__ src, long long N, long long ps,
                                                                double r, double half_r2, const Args<float> af,
                                                                double* __restrict__ partial) {
  using L = Lat<LAT>;
  constexpr int Q = L::Q;
  double acc[kRedVals] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const long long begin = (long long)blockIdx.x * kNaCellsPerBlock;
  const long long end = (begin + kNaCellsPerBlock < N) ? begin + kNaCellsPerBlock : N;
  for (long long cell = begin + threadIdx.x; cell < end; cell += kNaThreads) {
    static_for<Q>([&](auto I) {
      constexpr int i = decltype(I)::value;
      double gi, hi;
      decode_pair_d<Q, S>(src, i, ps, cell, L::grp(i), af, gi, hi);
      acc[0] += gi;
      if constexpr (L::cx(i) != 0) acc[1] += (r * L::cx(i)) * gi;
      if constexpr (L::cy(i) != 0) acc[2] += (r * L::cy(i)) * gi;
      if constexpr (L::cz(i) != 0) acc[3] += (r * L::cz(i)) * gi;
      acc[4] += half_r2 * L::c2(i) * gi + hi;
    });
  }
  __shared__ double sh[kNaThreads / 32][kRedVals];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kRedVals; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kRedVals) {
    double s = 0.0;
    for (int w = 0; w < kNaThreads / 32; ++w) s += sh[w][threadIdx.x];
    partial[blockIdx.x * kRedVals + threadIdx.x] = s;
  }
}

// Totals of the nblocks partials written by this call (one warp per value,
// fixed order).  Every slot read here was written earlier in the same call,
// so nothing has to be cleared between calls.
__global__ void k_conserve_chunk_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= kRedVals) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partial[b * kRedVals + k];
  s = warp_sum(s);
  if (lane == 0) out[k] = s;
}

template <int LAT, class S>
cudaError_t launch_chunk(const void* state, long long N, long long ps, double r, double half_r2,
                         const Args<float>& af, double* scratch, int nblocks, cudaStream_t st) {
  k_conserve_chunk<LAT, S><<<nblocks, kNaThreads, 0, st>>>(static_cast<const S*>(state), N, ps, r, half_r2, af,
                                                           scratch);
  return cudaGetLastError();
}

template <int LAT>
cudaError_t launch_chunk_prec(int prec, const void* state, long long N, long long ps, double r, double half_r2,
                              const Args<float>& af, double* scratch, int nblocks, cudaStream_t st) {
  switch (prec) {
    case kF64: return launch_chunk<LAT, double>(state, N, ps, r, half_r2, af, scratch, nblocks, st);
    case kF32: return launch_chunk<LAT, float>(state, N, ps, r, half_r2, af, scratch, nblocks, st);
    case kF32S16F: return launch_chunk<LAT, __half>(state, N, ps, r, half_r2, af, scratch, nblocks, st);
    case kF32S16BF: return launch_chunk<LAT, __nv_bfloat16>(state, N, ps, r, half_r2, af, scratch, nblocks, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" int lbm_conserved_noalloc(int lattice, int prec, double gamma, double rho0, double T0,
                                     const void* state, long long ncells, long long plane_stride, void* stream,
                                     double* out) {
  if (lattice != LBM_D2Q37 && lattice != LBM_D3Q107) return set_error(LBM_EINVAL, "unknown lattice");
  if (prec < kF64 || prec > kF32S16BF) return set_error(LBM_EINVAL, "unknown precision");
  if (!out) return set_error(LBM_EINVAL, "out is NULL");
  const int D = (lattice == LBM_D2Q37) ? 2 : 3;
  if (!(gamma > 1.0)) return set_error(LBM_EINVAL, "gamma must be > 1");
  double delta = 2.0 / (gamma - 1.0) - D;
  if (delta < -1e-12) return set_error(LBM_EINVAL, "gamma gives delta < 0 (gamma must be <= (D+2)/D)");
  if (delta < 0.0) delta = 0.0;
  // the reference state as lbm_create resolves it
  if (resolve_reference(prec, rho0, T0, &rho0, &T0) != LBM_OK)
    return set_error(LBM_EINVAL, "16-bit storage needs a positive reference density rho0");
  if (ncells < 0) return set_error(LBM_EINVAL, "ncells must be >= 0");
  if (ncells > kNaMaxCells)
    return set_error(LBM_EINVAL, "ncells exceeds the no-allocation maximum of 16777216 cells "
                                 "(4096 blocks of 4096 cells of static scratch); use lbm_conserved");
  if (plane_stride < ncells) return set_error(LBM_EINVAL, "plane_stride must be >= ncells");
  if (ncells > 0 && !state) return set_error(LBM_EINVAL, "state is NULL");
  if (ncells > 0) {
    // the kernels read whole storage words (8 bytes FP64, 4 bytes FP32 and
    // 16-bit pairs) from GPU memory of the current device: reject anything
    // else here instead of faulting on the GPU
    const size_t word = (prec == kF64) ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(state) % word != 0)
      return set_error(LBM_EINVAL, "state is not aligned to its " + std::to_string(word) + "-byte storage word");
    cudaPointerAttributes pa;
    cudaError_t e = cudaPointerGetAttributes(&pa, state);
    if (e != cudaSuccess) {
      cudaGetLastError();  // clear the error this query may leave
      return set_error(LBM_EINVAL, std::string("state is not a CUDA pointer: ") + cudaGetErrorString(e));
    }
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)
      return set_error(LBM_EINVAL, "state must be device or managed memory");
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(LBM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (pa.type == cudaMemoryTypeDevice && pa.device != dev)
      return set_error(LBM_EINVAL, "state lives on device " + std::to_string(pa.device) + ", not on the current device " +
                                       std::to_string(dev));
  }

  LatticeTable t;
  if (build_lattice_table(lattice, &t) != 0) return set_error(LBM_EINVAL, "lattice table refinement failed");
  // 16-bit codec constants of the reference equilibrium (rho0, u = 0, T0),
  // from the same helper the instances use
  Args<float> af{};
  double gref[10], pref[10], hscale[10];
  reference_constants(t, delta, rho0, T0, gref, pref, hscale);
  for (int g = 0; g < 10; ++g) {
    af.gref[g] = (float)gref[g];
    af.hscale[g] = (float)hscale[g];
  }

  double tmp[kRedVals] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (ncells > 0) {
    double* scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc != LBM_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nblocks = (int)((ncells + kNaCellsPerBlock - 1) / kNaCellsPerBlock);
    cudaError_t e = (lattice == LBM_D2Q37)
                        ? launch_chunk_prec<0>(prec, state, ncells, plane_stride, t.r, 0.5 * t.r * t.r, af, scratch,
                                               nblocks, st)
                        : launch_chunk_prec<1>(prec, state, ncells, plane_stride, t.r, 0.5 * t.r * t.r, af, scratch,
                                               nblocks, st);
    if (e == cudaSuccess) {
      k_conserve_chunk_final<<<1, 32 * kRedVals, 0, st>>>(scratch, nblocks, scratch + kNaMaxBlocks * kRedVals);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tmp, scratch + kNaMaxBlocks * kRedVals, sizeof(tmp), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(LBM_ECUDA, std::string("no-allocation reduction: ") + cudaGetErrorString(e));
  }
  // the state holds deviations from the reference equilibrium: add its totals
  const double Nd = (double)ncells;
  out[0] = Nd * rho0 + tmp[0];
  for (int a = 0; a < D; ++a) out[1 + a] = tmp[1 + a];
  out[1 + D] = Nd * rho0 * 0.5 * (D + delta) * T0 + tmp[4];
  return LBM_OK;
}
