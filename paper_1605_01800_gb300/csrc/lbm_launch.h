// Host-side launchers of the CUDA kernels (one translation unit per kernel
// family, so that the library builds in parallel).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

// CTA shapes of the step kernel: {TX threads in x, TYT threads in y, RY nodes
// per thread in y, minimum resident CTAs per SM}; the node tile is
// TX x (TYT * RY). Every shape computes bitwise the same result; they differ
// only in speed.
constexpr int kTileCount = 8;
constexpr int kTiles[kTileCount][4] = {
    {32, 8, 2, 4}, {32, 4, 2, 7}, {64, 4, 2, 4}, {32, 4, 4, 5},
    {32, 4, 4, 4}, {32, 4, 2, 8}, {32, 4, 2, 6}, {32, 8, 2, 3},
};

template <typename T>
struct StepArgs;
template <typename T>
struct PhysTable;
struct TileGrid;

// TMA-staged persistent FP32 variants (lbm_step_tma.cu); tile indices
// kTileCount .. kTileCount + tma_variant_count() - 1 of the public tile list.
// They take the tiles at least two cells away from every lattice edge (their
// boxes are plain rectangles of the lattice); the other tiles of the step go
// through the plain kernel of the same node tile (tma_plain_partner) in a
// second launch.
struct TmaArgs {
    const Tile* tiles;
    int n_tiles;
    const Geom* geom;
    const Phys<float>* phys;
    float* fout;               // buffer written this step (whole array)
    unsigned* status;
    long long wait_limit;      // clock cycles an mbarrier wait may take before the CTA gives up
    unsigned extra_tx;         // bytes added to every stage's expected count (0; tests only)
};
// Tensor maps travel as __grid_constant__ kernel parameters: per lattice the
// map of the buffer read this step and the map of its wall mask.
constexpr int kTmaMaxLattices = 64;
struct TmaMaps {
    CUtensorMap f[kTmaMaxLattices];
    CUtensorMap m[kTmaMaxLattices];
};
int tma_variant_count();
void tma_variant_shape(int v, int* tx, int* ty);
int tma_plain_partner(int v);
int tma_blocks_per_sm(int v);
cudaError_t launch_step_tma(int v, int grid, const TmaArgs& args, const TmaMaps& maps,
                            const PhysTable<float>& table, cudaStream_t s);
// Tensor maps of lattice g in both buffers (fmaps2[0..1]) and of its mask
// (mmap; zeroed when the lattice has no mask), boxes for a tx x ty tile.
bool encode_lattice_maps(const Geom& g, int tx, int ty, const float* buf0, const float* buf1,
                         const uint8_t* mask_base, CUtensorMap* fmaps2, CUtensorMap* mmap);

// Persistent software-pipelined FP32 variants (lbm_step_pipe.cu); tile
// indices kTileCount + tma_variant_count() + v. They take the full wall-free
// tiles (FastTile list); the other tiles of the step go through the plain
// kernel of the same node tile (pipe_plain_partner) in a second launch.
struct FastTile {
    long long f_off;       // plane 0 of the tile's lattice (element offset, both buffers)
    int plane, pitch, nx, ny;
    int lat, x0, y0, edge; // edge: within two cells of a lattice edge (wrapped pulls)
    int pad[2];
};
struct PipeArgs {
    const FastTile* fast;
    int n_fast;
    const Phys<float>* phys;   // used when the parameters do not travel as a kernel argument
    const float* fin;
    float* fout;
    unsigned* status;
};
int pipe_variant_count();
void pipe_variant_shape(int v, int* tx, int* ty);
int pipe_plain_partner(int v);
int pipe_blocks_per_sm(int v, bool table);
cudaError_t launch_step_pipe(int v, int grid, const PipeArgs& a, const PhysTable<float>* table, cudaStream_t s);

// table: the batch's parameters for the constant-bank path (batches of at
// most kParamLattices lattices), or null to read them from global memory.
// open: the batch holds lattices open in x (x-slabs); their kernels are
// instantiated apart from the ordinary ones.
// grid: the tile list as a regular grid (TileGrid::tiles_x > 0), which the
// shapes of four nodes per thread use to find tiles without their records;
// tiles_x = 0 otherwise (always for open batches and partial lists).
cudaError_t launch_step_f32_closed(int tile_index, int n_tiles, const StepArgs<float>& a,
                                   const PhysTable<float>* table, const TileGrid& grid, cudaStream_t s);
cudaError_t launch_step_f32_open(int tile_index, int n_tiles, const StepArgs<float>& a,
                                 const PhysTable<float>* table, const TileGrid& grid, cudaStream_t s);
inline cudaError_t launch_step_f32(int tile_index, int n_tiles, const StepArgs<float>& a,
                                   const PhysTable<float>* table, const TileGrid& grid, cudaStream_t s,
                                   bool open = false) {
    return open ? launch_step_f32_open(tile_index, n_tiles, a, table, grid, s)
                : launch_step_f32_closed(tile_index, n_tiles, a, table, grid, s);
}
cudaError_t launch_step_f64(int tile_index, int n_tiles, const StepArgs<double>& a, cudaStream_t s,
                            bool open = false);

// Lattices [lat0, lat0 + n_lat) of a context, for the FP64 helper kernels.
struct LaunchSet {
    const Geom* geoms;          // device array of every lattice's geometry
    const Phys<double>* phys;   // device array of every lattice's parameters
    const uint8_t* mask;        // device mask base (lattice rows at geom.mask_off)
    int lat0, n_lat;
    long long max_nodes;        // largest nx*ny among the lattices
    long long max_extent;       // largest nx + ny among the lattices
    int layout;                 // layout of the stored state (kLayoutPull, kLayoutNatural, kLayoutSwapped)
};

// Step of in-place storage: two launches over the plain kernel's tile list
// (tx x ty node tiles), psi of every node into `psi` (a plane per lattice in
// the stored layout, at f_off / 9, with a one-cell periodic frame), then the
// collision from `layout` (kLayoutNatural or kLayoutSwapped) into the other
// layout, in place.
cudaError_t launch_step_inplace_f32(const TileGeom* tg, int n_tiles, int tx, int ty, const Phys<float>* phys,
                                    float* f, const uint8_t* mask, float* psi, unsigned* status, int layout,
                                    cudaStream_t s);
cudaError_t launch_step_inplace_f64(const TileGeom* tg, int n_tiles, int tx, int ty, const Phys<double>* phys,
                                    double* f, const uint8_t* mask, double* psi, unsigned* status, int layout,
                                    cudaStream_t s);

// Initial state: f_a such that the next pull gathers f_eq(rho, u) at every
// fluid node. rho/ux/uy are device arrays indexed by geom.node_off + y*nx + x
// (ux/uy may be null for u = 0). bad[lat] is set to gen for invalid input
// (bad: a device-visible address, e.g. mapped page-locked host memory).
cudaError_t launch_init_f32(const LaunchSet& L, const double* rho, const double* ux,
                            const double* uy, float* f, unsigned* bad, unsigned gen, cudaStream_t s);
cudaError_t launch_init_f64(const LaunchSet& L, const double* rho, const double* ux,
                            const double* uy, double* f, unsigned* bad, unsigned gen, cudaStream_t s);

// Initial state of one lattice open in x (an x-slab): rho/ux/uy are device
// arrays of (nx + 2) x ny values, the neighbouring slabs' edge columns
// included (ux/uy may be null); `mask` is the device mask base.
cudaError_t launch_init_open_f32(const Geom& g, double rho_ref, const double* rho, const double* ux,
                                 const double* uy, const uint8_t* mask, float* f, unsigned* bad, int lat,
                                 unsigned gen, cudaStream_t s);
cudaError_t launch_init_open_f64(const Geom& g, double rho_ref, const double* rho, const double* ux,
                                 const double* uy, const uint8_t* mask, double* f, unsigned* bad, int lat,
                                 unsigned gen, cudaStream_t s);
// Halo of an x-slab (12 * ny values): pack what the neighbour on `side` reads
// from the state `f` into `buf`, or unpack a neighbour's halo from `buf`
// into the frame of `f` (pack = false).
cudaError_t launch_halo_f32(const Geom& g, float* f, int side, float* buf, bool pack, cudaStream_t s);
cudaError_t launch_halo_f64(const Geom& g, double* f, int side, double* buf, bool pack, cudaStream_t s);

// rho, v (Eq. 6), p (Eq. 10) into device arrays indexed like the init inputs
// (all four required), computed in FP64 from the stored distribution; psi is
// scratch of one plane per lattice in the stored layout (element offset
// f_off / 9), its frame holding the psi of the periodic neighbours.
cudaError_t launch_moments_f32(const LaunchSet& L, const float* f, double* psi, double* rho, double* ux,
                               double* uy, double* p, cudaStream_t s);
cudaError_t launch_moments_f64(const LaunchSet& L, const double* f, double* psi, double* rho, double* ux,
                               double* uy, double* p, cudaStream_t s);

// rho alone (the first output of launch_moments_*, same values).
cudaError_t launch_density_f32(const LaunchSet& L, const float* f, double* rho, cudaStream_t s);
cudaError_t launch_density_f64(const LaunchSet& L, const double* f, double* rho, cudaStream_t s);

// Fixed-order FP64 mass of one lattice: sum over fluid nodes of the stored
// values plus rho_ref * n_fluid. `partials` is scratch of kMassBlocks doubles.
constexpr int kMassBlocks = 120;
constexpr int kMassThreads = 256;
cudaError_t launch_mass_f32(const Geom& g, double rho_ref, long long n_fluid, const float* f,
                            const uint8_t* mask, int layout, double* partials, double* out, cudaStream_t s);
cudaError_t launch_mass_f64(const Geom& g, double rho_ref, long long n_fluid, const double* f,
                            const uint8_t* mask, int layout, double* partials, double* out, cudaStream_t s);

// Fixed-order FP64 totals of the lattices of L: out[3k .. 3k + 2] = mass (the
// value launch_mass_* gives, bit for bit), sum of j_x + F_x/2, sum of j_y +
// F_y/2 over the fluid nodes of lattice L.lat0 + k. psi, rho, jx, jy are the
// read-out scratch of launch_moments_*; partials holds 4 * kMassBlocks
// doubles per lattice.
cudaError_t launch_totals_f32(const LaunchSet& L, const float* f, double* psi, double* rho, double* jx,
                              double* jy, double* partials, double* out, cudaStream_t s);
cudaError_t launch_totals_f64(const LaunchSet& L, const double* f, double* psi, double* rho, double* jx,
                              double* jy, double* partials, double* out, cudaStream_t s);

}  // namespace lbm
