// Kernel instantiations and launchers of one (lattice, precision) pair,
// selected at compile time by LBM_LAT (0 = D2Q37, 1 = D3Q107) and LBM_PREC
// (0 = FP64, 1 = FP32, 2 = FP32 compute / FP16 storage, 3 = FP32 / BF16).
// The build compiles this file once per pair so the objects build in parallel.
#include "fd_march.cuh"

#ifndef LBM_LAT
#error "LBM_LAT must be defined"
#endif
#ifndef LBM_PREC
#error "LBM_PREC must be defined"
#endif

namespace lbm {

#if LBM_PREC == 0
using StoreT = double;
using ComputeT = double;
#elif LBM_PREC == 1
using StoreT = float;
using ComputeT = float;
#elif LBM_PREC == 2
using StoreT = __half;
using ComputeT = float;
#else
using StoreT = __nv_bfloat16;
using ComputeT = float;
#endif

#define LBM_CAT2(a, b, c) a##_##b##_##c
#define LBM_CAT(a, b, c) LBM_CAT2(a, b, c)

extern const Launchers LBM_CAT(kLaunchers, LBM_LAT, LBM_PREC) = {
    &launch_step_plain<LBM_LAT, StoreT, ComputeT>,
    &launch_init_t<LBM_LAT, StoreT, ComputeT>,
    &launch_moments_t<LBM_LAT, StoreT, ComputeT>,
    &launch_conserve_t<LBM_LAT, StoreT>,
    &launch_pool_step_t<LBM_LAT, StoreT, ComputeT>,
    &launch_pool_advance_t<ComputeT>,
    &pool_grid_t<LBM_LAT, StoreT, ComputeT>,
    pool_tile_cells<LBM_LAT, StoreT>(),
    &shape_count_t<LBM_LAT, StoreT>,
    &shape_get_t<LBM_LAT, StoreT>,
    &configure_step_t<LBM_LAT, StoreT, ComputeT>,
    &launch_step_fd_any<LBM_LAT, StoreT, ComputeT>,
};

}  // namespace lbm
