// FP32 instantiations of the fused step kernel (deviation or plain storage).
#include "lbm_launch.h"
#include "lbm_step.cuh"

namespace lbm {

template <int TX, int TYT, int RY, int MINB, bool TABLE>
static cudaError_t launch_tile(int n_tiles, const StepArgs<float>& a, const PhysTable<float>* table,
                               cudaStream_t s) {
    TableOf<float, TABLE> t{};
    if constexpr (TABLE) t = *table;
    step_kernel<float, TX, TYT, RY, MINB, TABLE><<<n_tiles, dim3(TX, TYT), 0, s>>>(a, t);
    return cudaGetLastError();
}

cudaError_t launch_step_f32(int tile_index, int n_tiles, const StepArgs<float>& args,
                            const PhysTable<float>* table, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    switch (tile_index) {
    case 0: return table ? launch_tile<32, 8, 2, 4, true>(n_tiles, args, table, s)
                   : launch_tile<32, 8, 2, 4, false>(n_tiles, args, nullptr, s);
    case 1: return table ? launch_tile<32, 4, 2, 7, true>(n_tiles, args, table, s)
                   : launch_tile<32, 4, 2, 7, false>(n_tiles, args, nullptr, s);
    case 2: return table ? launch_tile<64, 4, 2, 4, true>(n_tiles, args, table, s)
                   : launch_tile<64, 4, 2, 4, false>(n_tiles, args, nullptr, s);
    case 3: return table ? launch_tile<32, 4, 4, 5, true>(n_tiles, args, table, s)
                   : launch_tile<32, 4, 4, 5, false>(n_tiles, args, nullptr, s);
    case 4: return table ? launch_tile<32, 4, 4, 4, true>(n_tiles, args, table, s)
                   : launch_tile<32, 4, 4, 4, false>(n_tiles, args, nullptr, s);
    case 5: return table ? launch_tile<32, 4, 2, 8, true>(n_tiles, args, table, s)
                   : launch_tile<32, 4, 2, 8, false>(n_tiles, args, nullptr, s);
    case 6: return table ? launch_tile<32, 4, 2, 6, true>(n_tiles, args, table, s)
                   : launch_tile<32, 4, 2, 6, false>(n_tiles, args, nullptr, s);
    case 7: return table ? launch_tile<32, 8, 2, 3, true>(n_tiles, args, table, s)
                   : launch_tile<32, 8, 2, 3, false>(n_tiles, args, nullptr, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
