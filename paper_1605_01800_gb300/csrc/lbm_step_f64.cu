// FP64 instantiations of the fused step kernel (plain FP64 storage and arithmetic).
#include "lbm_launch.h"
#include "lbm_step.cuh"

namespace lbm {

template <int TX, int TYT, int RY, bool OPEN>
static cudaError_t launch_tile(int n_tiles, const StepArgs<double>& a, cudaStream_t s) {
    step_kernel<double, TX, TYT, RY, 1, false, OPEN><<<n_tiles, dim3(TX, TYT), 0, s>>>(a, NoTable{0});
    return cudaGetLastError();
}

template <bool OPEN>
static cudaError_t launch_shape(int tile_index, int n_tiles, const StepArgs<double>& args, cudaStream_t s) {
    switch (tile_index) {
    case 0: case 7: return launch_tile<32, 8, 2, OPEN>(n_tiles, args, s);
    case 1: case 5: case 6: return launch_tile<32, 4, 2, OPEN>(n_tiles, args, s);
    case 2: return launch_tile<64, 4, 2, OPEN>(n_tiles, args, s);
    case 3: case 4: return launch_tile<32, 4, 4, OPEN>(n_tiles, args, s);
    default: return cudaErrorInvalidValue;
    }
}

// open: the batch holds lattices open in x (see tile_general)
cudaError_t launch_step_f64(int tile_index, int n_tiles, const StepArgs<double>& args, cudaStream_t s,
                            bool open) {
    if (n_tiles <= 0) return cudaSuccess;
    return open ? launch_shape<true>(tile_index, n_tiles, args, s) : launch_shape<false>(tile_index, n_tiles, args, s);
}

}  // namespace lbm
