// Internal runtime of the library: the instance record and the launchers
// that each lattice's translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/lbm.h"
#include "kernels.cuh"
#include "lattice.h"

namespace lbm {

enum Prec { kF64 = 0, kF32 = 1, kF32S16F = 2, kF32S16BF = 3 };

// Kernel launch shape of the step, per (lattice, precision); chosen by the
// built-in defaults or the autotuner.
struct StepShape {
  int index;  // candidate index of the (lattice, storage) shape table (launch_impl.cuh)
};

struct Instance {
  int lattice, prec, D, Q, G;
  int n[3], bc[3];
  long long N;         // cells
  long long ps;        // plane stride (elements), N rounded up to 64
  size_t word;         // bytes per stored population
  size_t buf_bytes;    // bytes of one population buffer (2Q planes)
  cudaStream_t stream;
  unsigned char* mem;  // base of the device allocation
  bool own_mem;
  void* buf[2];        // population buffers
  int cur;             // buffer holding the current state
  unsigned int* flag;  // device error word
  double* red_out;     // device: final conservation sums (kRedVals)
  double* red_partial; // device: per-block partials (kRedMaxBlocks * kRedVals)
  LatticeTable table;
  double gamma, delta, tau_f, tau_g, rho0, T0;
  long steps_done;
  Args<double> ad;
  Args<float> af;
  StepShape shape;
  int fd_kernel;  // finite-difference step kernel: LBM_FD_AUTO / LBM_FD_CELL / LBM_FD_MARCH
  // CUDA graph of `graph_steps` consecutive steps (even, so the buffers are
  // back in place after a replay); 0 = plain launches
  int graph_steps;
  int graph_shape;           // shape index the graph was captured with
  cudaGraphExec_t graph_exec;
  cudaGraph_t graph;
};

// Bytes of the tail region after the two buffers.
constexpr size_t kTailBytes = 256 /*flag*/ + 256 /*red_out*/ + sizeof(double) * kRedMaxBlocks * kRedVals;

inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Arguments of the pool launchers (device pointers of the pool tables).
struct PoolLaunch {
  void* slots;          // PoolSlot<C>[nslots]
  const int4* tiles;    // tile list: slot, x0, y, z
  const int* ntiles;    // device: tiles in the list
  int nslots;
  int grid;             // persistent grid of the batched step
  cudaStream_t stream;
};

// Launchers of one (lattice, precision) pair; each pair is compiled as its
// own object from step_inst.cu.  All launch on inst->stream and return the
// CUDA error of the launch.
struct Launchers {
  cudaError_t (*step)(const Instance* inst, const void* src, void* dst);
  cudaError_t (*init)(const Instance* inst, void* dst, const double* rho, const double* u, const double* T);
  cudaError_t (*moments)(const Instance* inst, const void* src, double* rho, double* u, double* T);
  cudaError_t (*conserve)(const Instance* inst, const void* src, double* partial, int nblocks);
  cudaError_t (*pool_step)(const PoolLaunch& pl);
  cudaError_t (*pool_advance)(const PoolLaunch& pl);
  int (*pool_grid)();
  int pool_tile_cells;  // cells per tile along x
  int (*shape_count)();
  void (*shape_get)(int k, int* stage, int* bx);
  cudaError_t (*configure)(const Instance* inst);
  cudaError_t (*step_fd)(const Instance* inst, const void* src, void* dst, double lam);
};

extern const Launchers kLaunchers_0_0, kLaunchers_0_1, kLaunchers_0_2, kLaunchers_0_3;
extern const Launchers kLaunchers_1_0, kLaunchers_1_1, kLaunchers_1_2, kLaunchers_1_3;

StepShape default_shape(int lattice, int prec);

// Records msg as this thread's lbm_last_error() and returns code.
int set_error(int code, const std::string& msg);


// Validates the parameters of an instance and fills everything but its
// memory (buffers, flag, reduction scratch) and its Args; returns a status.
int prepare_instance(Instance* I, int lattice, double gamma, double tau_f, double tau_g, const lbm_grid* grid);
// Fills I->ad and I->af from the instance (after its flag pointer is set).
void fill_instance_args(Instance* I);
// The reference state an instance of precision prec stores its populations
// against, from the caller's (rho0, T0): rho0 > 0 is taken as given; rho0 < 0
// asks for whole storage (*rho0_out = 0, FP64 and FP32 storage only); 0 or
// NaN is the precision's default, whole storage for FP64 and rho0 = 1 for
// FP32 and 16-bit storage.  T0 that is not positive (NaN included) is 1.
// Returns LBM_OK or LBM_EINVAL (whole storage asked for 16-bit storage).
int resolve_reference(int prec, double rho0, double T0, double* rho0_out, double* T0_out);
// Reference equilibrium per velocity group at (rho0, u = 0, T0), Eq. (18):
// gref[g], pref[g] = gref / (w rho0) - 1, and the scale hscale[g] of the
// 16-bit h codec (groups past t.G get 1, 0, 1).
void reference_constants(const LatticeTable& t, double delta, double rho0, double T0, double* gref,
                         double* pref, double* hscale);
// Bytes of one population buffer (2Q planes, 256-byte rounded).
size_t instance_buffer_bytes(int Q, long long N, int prec);
const Launchers& launchers_for(int lattice, int prec);

}  // namespace lbm
