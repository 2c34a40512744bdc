// FP64 instantiations of the fused step kernel (plain FP64 storage and arithmetic).
#include "lbm_launch.h"
#include "lbm_step.cuh"

namespace lbm {

template <int TX, int TYT, int RY>
static cudaError_t launch_tile(int n_tiles, const StepArgs<double>& a, cudaStream_t s) {
    step_kernel<double, TX, TYT, RY, 1, false><<<n_tiles, dim3(TX, TYT), 0, s>>>(a, NoTable{0});
    return cudaGetLastError();
}

cudaError_t launch_step_f64(int tile_index, int n_tiles, const StepArgs<double>& args, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    switch (tile_index) {
    case 0: return launch_tile<32, 8, 2>(n_tiles, args, s);
    case 1: return launch_tile<32, 4, 2>(n_tiles, args, s);
    case 2: return launch_tile<64, 4, 2>(n_tiles, args, s);
    case 3: return launch_tile<32, 4, 4>(n_tiles, args, s);
    case 4: return launch_tile<32, 4, 4>(n_tiles, args, s);
    case 5: return launch_tile<32, 4, 2>(n_tiles, args, s);
    case 6: return launch_tile<32, 4, 2>(n_tiles, args, s);
    case 7: return launch_tile<32, 8, 2>(n_tiles, args, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
