// Non-hot kernels of the library: initial state, macroscopic read-out and the
// FP64 mass reduction. All arithmetic here is FP64.
#include "lbm_launch.h"

namespace lbm {

namespace {

__constant__ int kEx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kEy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__constant__ int kOpp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
__constant__ double kWeq[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                               1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

__device__ __forceinline__ bool is_solid(const uint8_t* mask, const Geom& g, int x, int y) {
    return mask != nullptr && mask[node_index(g, x, y)] != 0;
}

// Second-order equilibrium in velocity space, f_eq_a = w_a rho (1 + 3 e.u +
// 9/2 (e.u)^2 - 3/2 u^2), whose moments are Eq. 4.
__device__ __forceinline__ double feq(int a, double rho, double ux, double uy) {
    const double eu = kEx[a] * ux + kEy[a] * uy;
    return kWeq[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * (ux * ux + uy * uy));
}

// The step kernel pulls f_a(x) = fstored_a(x - e_a), or fstored_abar(x) when
// x - e_a is solid. To make that pull return f_eq at every fluid node, the
// stored value at node y for population b is f_eq_b of the node y + e_b it
// streams into, or f_eq_bbar(y) when y + e_b is solid (the reflected link).
template <typename T>
__global__ void init_kernel(const Geom* __restrict__ geoms, const Phys<double>* __restrict__ phys,
                            int lat0, const double* __restrict__ rho, const double* __restrict__ ux,
                            const double* __restrict__ uy, const uint8_t* __restrict__ mask_base,
                            T* __restrict__ f_base) {
    const int lat = lat0 + blockIdx.y;
    const Geom g = geoms[lat];
    const double rho_ref = phys[lat].rho_ref;
    const uint8_t* mask = g.has_mask ? mask_base + g.mask_off : nullptr;
    T* f = f_base + g.f_off;
    rho += g.node_off;
    if (ux) ux += g.node_off;
    if (uy) uy += g.node_off;
    const long long n = (long long)g.nx * g.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)(i / g.nx);
        T out[9];
        if (is_solid(mask, g, x, y)) {
            for (int b = 0; b < 9; ++b) out[b] = T(0);
            store_node<T>(f, g, x, y, out);
            continue;
        }
        for (int b = 0; b < 9; ++b) {
            const int xt = wrap_index(x + kEx[b], g.nx), yt = wrap_index(y + kEy[b], g.ny);
            double v;
            if (is_solid(mask, g, xt, yt)) {
                v = feq(kOpp[b], rho[i], ux ? ux[i] : 0.0, uy ? uy[i] : 0.0);
            } else {
                const long long j = (long long)yt * g.nx + xt;
                v = feq(b, rho[j], ux ? ux[j] : 0.0, uy ? uy[j] : 0.0);
            }
            out[b] = (T)(v - kWeq[b] * rho_ref);
        }
        store_node<T>(f, g, x, y, out);
    }
}

// Pulled distribution of node (x, y) as FP64 full populations; false if solid.
template <typename T>
__device__ __forceinline__ bool pulled_fp64(const Geom& g, const T* f, const uint8_t* mask,
                                            double rho_ref, int x, int y, double out[9]) {
    T tmp[9];
    if (pull_node<T>(f, mask, (int)g.plane, g.pitch, node_index(g, x, y), tmp)) return false;
    for (int a = 0; a < 9; ++a) out[a] = (double)tmp[a] + kWeq[a] * rho_ref;
    return true;
}

__device__ __forceinline__ double psi_fp64(double rho, const Phys<double>& P) {
    unsigned unused = 0;
    return psi_of(rho, P, unused);
}

template <typename T>
__global__ void moments_kernel(const Geom* __restrict__ geoms, const Phys<double>* __restrict__ phys,
                               int lat0, const T* __restrict__ f_base,
                               const uint8_t* __restrict__ mask_base, double* __restrict__ rho_out,
                               double* __restrict__ ux_out, double* __restrict__ uy_out,
                               double* __restrict__ p_out) {
    const int lat = lat0 + blockIdx.y;
    const Geom g = geoms[lat];
    const Phys<double> P = phys[lat];
    const uint8_t* mask = g.has_mask ? mask_base + g.mask_off : nullptr;
    const T* f = f_base + g.f_off;
    const long long n = (long long)g.nx * g.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long o = g.node_off + i;
        const int x = (int)(i % g.nx), y = (int)(i / g.nx);
        double fc[9];
        if (!pulled_fp64<T>(g, f, mask, P.rho_ref, x, y, fc)) {
            if (rho_out) rho_out[o] = 0.0;
            if (ux_out) ux_out[o] = 0.0;
            if (uy_out) uy_out[o] = 0.0;
            if (p_out) p_out[o] = 0.0;
            continue;
        }
        double rho = 0.0, jx = 0.0, jy = 0.0;
        for (int a = 0; a < 9; ++a) {
            rho += fc[a];
            jx += kEx[a] * fc[a];
            jy += kEy[a] * fc[a];
        }
        const double psi = psi_fp64(rho, P);
        double gx = 0.0, gy = 0.0;
        for (int a = 1; a < 9; ++a) {
            const int xn = x + kEx[a], yn = y + kEy[a];  // ghost frame covers -1 and n
            double fn[9];
            double pn = psi;  // solid neighbour: the node's own psi
            if (pulled_fp64<T>(g, f, mask, P.rho_ref, xn, yn, fn)) {
                double rn = 0.0;
                for (int b = 0; b < 9; ++b) rn += fn[b];
                pn = psi_fp64(rn, P);
            }
            const double w = (a < 5) ? (1.0 / 3.0) : (1.0 / 12.0);
            gx += w * pn * kEx[a];
            gy += w * pn * kEy[a];
        }
        const double Fx = -P.G * psi * gx, Fy = -P.G * psi * gy;
        if (rho_out) rho_out[o] = rho;
        if (ux_out) ux_out[o] = (jx + 0.5 * Fx) / rho;
        if (uy_out) uy_out[o] = (jy + 0.5 * Fy) / rho;
        // Eq. 10: p = rho c_s^2 + G c^2 psi^2 / 2
        if (p_out) p_out[o] = rho * P.cs2 + 0.5 * P.G * psi * psi;
    }
}

// Partial sums: block b adds the stored values of the fluid nodes i = b*T + t
// + k*B*T in a fixed order, then a fixed tree inside the block.
template <typename T>
__global__ void mass_partial_kernel(Geom g, const T* __restrict__ f, const uint8_t* __restrict__ mask,
                                    double* __restrict__ partials) {
    __shared__ double red[kMassThreads];
    const long long n = (long long)g.nx * g.ny;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)kMassThreads + threadIdx.x; i < n;
         i += (long long)kMassBlocks * kMassThreads) {
        const int x = (int)(i % g.nx), y = (int)(i / g.nx);
        if (is_solid(mask, g, x, y)) continue;
        const long long c = node_index(g, x, y);
        double s = 0.0;
        for (int a = 0; a < 9; ++a) s += (double)f[a * g.plane + c];
        acc += s;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kMassThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void mass_final_kernel(const double* __restrict__ partials, double rho_ref,
                                  long long n_fluid, double* out) {
    double s = 0.0;
    for (int b = 0; b < kMassBlocks; ++b) s += partials[b];
    *out = s + rho_ref * (double)n_fluid;
}

// Rewrite every lattice's ghost frame from the nodes it images (after the
// node values were written by a copy, e.g. when a checkpoint is loaded).
template <typename T>
__global__ void ghost_refresh_kernel(const Geom* __restrict__ geoms, int lat0, T* __restrict__ f_base) {
    const int lat = lat0 + blockIdx.y;
    const Geom g = geoms[lat];
    T* f = f_base + g.f_off;
    const long long n = (long long)g.nx * g.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)(i / g.nx);
        if (!(x < 2 || x >= g.nx - 2 || y < 2 || y >= g.ny - 2)) continue;
        T v[9];
        const int c = node_index(g, x, y);
        for (int a = 0; a < 9; ++a) v[a] = f[a * g.plane + c];
        store_ghost_images<T>(f, g, x, y, v);
    }
}

dim3 lattice_grid(long long max_nodes, int n_lat, int threads) {
    long long bx = (max_nodes + threads - 1) / threads;
    if (bx > 4096) bx = 4096;
    if (bx < 1) bx = 1;
    return dim3((unsigned)bx, (unsigned)n_lat);
}

template <typename T>
cudaError_t init_impl(const LaunchSet& L, const double* rho, const double* ux, const double* uy,
                      T* f, cudaStream_t s) {
    init_kernel<T><<<lattice_grid(L.max_nodes, L.n_lat, 256), 256, 0, s>>>(
        L.geoms, L.phys, L.lat0, rho, ux, uy, L.mask, f);
    return cudaGetLastError();
}

template <typename T>
cudaError_t moments_impl(const LaunchSet& L, const T* f, double* rho, double* ux, double* uy,
                         double* p, cudaStream_t s) {
    moments_kernel<T><<<lattice_grid(L.max_nodes, L.n_lat, 128), 128, 0, s>>>(
        L.geoms, L.phys, L.lat0, f, L.mask, rho, ux, uy, p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mass_impl(const Geom& g, double rho_ref, long long n_fluid, const T* f,
                      const uint8_t* mask, double* partials, double* out, cudaStream_t s) {
    mass_partial_kernel<T><<<kMassBlocks, kMassThreads, 0, s>>>(g, f + g.f_off, mask, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mass_final_kernel<<<1, 1, 0, s>>>(partials, rho_ref, n_fluid, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t ghost_impl(const LaunchSet& L, T* f, cudaStream_t s) {
    ghost_refresh_kernel<T><<<lattice_grid(L.max_nodes, L.n_lat, 256), 256, 0, s>>>(L.geoms, L.lat0, f);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ghost_refresh_f32(const LaunchSet& L, float* f, cudaStream_t s) {
    return ghost_impl<float>(L, f, s);
}
cudaError_t launch_ghost_refresh_f64(const LaunchSet& L, double* f, cudaStream_t s) {
    return ghost_impl<double>(L, f, s);
}

cudaError_t launch_init_f32(const LaunchSet& L, const double* rho, const double* ux,
                            const double* uy, float* f, cudaStream_t s) {
    return init_impl<float>(L, rho, ux, uy, f, s);
}
cudaError_t launch_init_f64(const LaunchSet& L, const double* rho, const double* ux,
                            const double* uy, double* f, cudaStream_t s) {
    return init_impl<double>(L, rho, ux, uy, f, s);
}
cudaError_t launch_moments_f32(const LaunchSet& L, const float* f, double* rho, double* ux,
                               double* uy, double* p, cudaStream_t s) {
    return moments_impl<float>(L, f, rho, ux, uy, p, s);
}
cudaError_t launch_moments_f64(const LaunchSet& L, const double* f, double* rho, double* ux,
                               double* uy, double* p, cudaStream_t s) {
    return moments_impl<double>(L, f, rho, ux, uy, p, s);
}
cudaError_t launch_mass_f32(const Geom& g, double rho_ref, long long n_fluid, const float* f,
                            const uint8_t* mask, double* partials, double* out, cudaStream_t s) {
    return mass_impl<float>(g, rho_ref, n_fluid, f, mask, partials, out, s);
}
cudaError_t launch_mass_f64(const Geom& g, double rho_ref, long long n_fluid, const double* f,
                            const uint8_t* mask, double* partials, double* out, cudaStream_t s) {
    return mass_impl<double>(g, rho_ref, n_fluid, f, mask, partials, out, s);
}

}  // namespace lbm
