// Host-side launchers of the CUDA kernels (one translation unit per kernel
// family, so that the library builds in parallel).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

// CTA tiles of the step kernel: {TX, TY}. Every tile computes bitwise the same
// result; they differ only in speed.
constexpr int kTileCount = 7;
constexpr int kTiles[kTileCount][2] = {
    {32, 8}, {64, 4}, {32, 16}, {128, 2}, {64, 8}, {128, 4}, {16, 16},
};

template <typename T>
struct StepArgs;

cudaError_t launch_step_f32(int tile_index, int n_tiles, const StepArgs<float>& a, cudaStream_t s);
cudaError_t launch_step_f64(int tile_index, int n_tiles, const StepArgs<double>& a, cudaStream_t s);

// Initial state: f_a such that the next pull gathers f_eq(rho, u) at every
// fluid node. rho/ux/uy are device arrays of nx*ny doubles (ux/uy may be null).
cudaError_t launch_init_f32(const Geom& g, float rho_ref, const double* rho, const double* ux,
                            const double* uy, const uint8_t* mask, float* f, cudaStream_t s);
cudaError_t launch_init_f64(const Geom& g, double rho_ref, const double* rho, const double* ux,
                            const double* uy, const uint8_t* mask, double* f, cudaStream_t s);

// rho, v (Eq. 6), p (Eq. 10) of one lattice into device arrays of nx*ny
// doubles (any may be null), computed in FP64 from the stored distribution.
cudaError_t launch_moments_f32(const Geom& g, const Phys<double>& P, const float* f,
                               const uint8_t* mask, double* rho, double* ux, double* uy,
                               double* p, cudaStream_t s);
cudaError_t launch_moments_f64(const Geom& g, const Phys<double>& P, const double* f,
                               const uint8_t* mask, double* rho, double* ux, double* uy,
                               double* p, cudaStream_t s);

// Fixed-order FP64 mass of one lattice: sum over fluid nodes of the stored
// values plus rho_ref * n_fluid. `partials` is scratch of kMassBlocks doubles.
constexpr int kMassBlocks = 120;
constexpr int kMassThreads = 256;
cudaError_t launch_mass_f32(const Geom& g, double rho_ref, long long n_fluid, const float* f,
                            const uint8_t* mask, double* partials, double* out, cudaStream_t s);
cudaError_t launch_mass_f64(const Geom& g, double rho_ref, long long n_fluid, const double* f,
                            const uint8_t* mask, double* partials, double* out, cudaStream_t s);

}  // namespace lbm
