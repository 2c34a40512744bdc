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

__device__ __forceinline__ bool is_solid(const uint8_t* mask, int pitch, int x, int y) {
    return mask != nullptr && mask[y * pitch + x] != 0;
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
__global__ void init_kernel(Geom g, T rho_ref, const double* __restrict__ rho,
                            const double* __restrict__ ux, const double* __restrict__ uy,
                            const uint8_t* __restrict__ mask, T* __restrict__ f) {
    const long long n = (long long)g.nx * g.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)(i / g.nx);
        const long long c = (long long)y * g.pitch + x;
        if (is_solid(mask, g.pitch, x, y)) {
            for (int b = 0; b < 9; ++b) f[b * g.plane + c] = T(0);
            continue;
        }
        for (int b = 0; b < 9; ++b) {
            const int xt = wrap_index(x + kEx[b], g.nx), yt = wrap_index(y + kEy[b], g.ny);
            double v;
            if (is_solid(mask, g.pitch, xt, yt)) {
                v = feq(kOpp[b], rho[i], ux ? ux[i] : 0.0, uy ? uy[i] : 0.0);
            } else {
                const long long j = (long long)yt * g.nx + xt;
                v = feq(b, rho[j], ux ? ux[j] : 0.0, uy ? uy[j] : 0.0);
            }
            f[b * g.plane + c] = (T)(v - kWeq[b] * (double)rho_ref);
        }
    }
}

// Pulled distribution of node (x, y) as FP64 full populations; false if solid.
template <typename T>
__device__ __forceinline__ bool pulled_fp64(const Geom& g, const T* f, const uint8_t* mask,
                                            double rho_ref, int x, int y, double out[9]) {
    T tmp[9];
    if (pull_node<T>(f, mask, (int)g.plane, g.pitch, g.nx, g.ny, x, y, tmp)) return false;
    for (int a = 0; a < 9; ++a) out[a] = (double)tmp[a] + kWeq[a] * rho_ref;
    return true;
}

__device__ __forceinline__ double psi_fp64(double rho, const Phys<double>& P) {
    unsigned unused = 0;
    return psi_of(rho, P, unused);
}

template <typename T>
__global__ void moments_kernel(Geom g, Phys<double> P, const T* __restrict__ f,
                               const uint8_t* __restrict__ mask, double* __restrict__ rho_out,
                               double* __restrict__ ux_out, double* __restrict__ uy_out,
                               double* __restrict__ p_out) {
    const long long n = (long long)g.nx * g.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)(i / g.nx);
        double fc[9];
        if (!pulled_fp64<T>(g, f, mask, P.rho_ref, x, y, fc)) {
            if (rho_out) rho_out[i] = 0.0;
            if (ux_out) ux_out[i] = 0.0;
            if (uy_out) uy_out[i] = 0.0;
            if (p_out) p_out[i] = 0.0;
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
            const int xn = wrap_index(x + kEx[a], g.nx), yn = wrap_index(y + kEy[a], g.ny);
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
        if (rho_out) rho_out[i] = rho;
        if (ux_out) ux_out[i] = (jx + 0.5 * Fx) / rho;
        if (uy_out) uy_out[i] = (jy + 0.5 * Fy) / rho;
        // Eq. 10: p = rho c_s^2 + G c^2 psi^2 / 2
        if (p_out) p_out[i] = rho * P.cs2 + 0.5 * P.G * psi * psi;
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
        if (is_solid(mask, g.pitch, x, y)) continue;
        const long long c = (long long)y * g.pitch + x;
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

template <typename T>
cudaError_t init_impl(const Geom& g, T rho_ref, const double* rho, const double* ux,
                      const double* uy, const uint8_t* mask, T* f, cudaStream_t s) {
    const long long n = (long long)g.nx * g.ny;
    const int threads = 256;
    const int blocks = (int)((n + threads - 1) / threads < 65535 ? (n + threads - 1) / threads : 65535);
    init_kernel<T><<<blocks, threads, 0, s>>>(g, rho_ref, rho, ux, uy, mask, f + g.f_off);
    return cudaGetLastError();
}

template <typename T>
cudaError_t moments_impl(const Geom& g, const Phys<double>& P, const T* f, const uint8_t* mask,
                         double* rho, double* ux, double* uy, double* p, cudaStream_t s) {
    const long long n = (long long)g.nx * g.ny;
    const int threads = 128;
    const int blocks = (int)((n + threads - 1) / threads < 65535 ? (n + threads - 1) / threads : 65535);
    moments_kernel<T><<<blocks, threads, 0, s>>>(g, P, f + g.f_off, mask, rho, ux, uy, p);
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

}  // namespace

cudaError_t launch_init_f32(const Geom& g, float rho_ref, const double* rho, const double* ux,
                            const double* uy, const uint8_t* mask, float* f, cudaStream_t s) {
    return init_impl<float>(g, rho_ref, rho, ux, uy, mask, f, s);
}
cudaError_t launch_init_f64(const Geom& g, double rho_ref, const double* rho, const double* ux,
                            const double* uy, const uint8_t* mask, double* f, cudaStream_t s) {
    return init_impl<double>(g, rho_ref, rho, ux, uy, mask, f, s);
}
cudaError_t launch_moments_f32(const Geom& g, const Phys<double>& P, const float* f,
                               const uint8_t* mask, double* rho, double* ux, double* uy,
                               double* p, cudaStream_t s) {
    return moments_impl<float>(g, P, f, mask, rho, ux, uy, p, s);
}
cudaError_t launch_moments_f64(const Geom& g, const Phys<double>& P, const double* f,
                               const uint8_t* mask, double* rho, double* ux, double* uy,
                               double* p, cudaStream_t s) {
    return moments_impl<double>(g, P, f, mask, rho, ux, uy, p, s);
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
