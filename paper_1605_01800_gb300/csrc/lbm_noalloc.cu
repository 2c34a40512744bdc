// Mass reduction that allocates no memory: the per-block partial sums live in
// a fixed file-scope device array instead of memory obtained from cudaMalloc.
//
// Some callers cannot allocate device memory at the point where they want a
// mass check: applications whose own allocator owns all device memory and
// hands out none, or real-time loops that must not stall in the driver's
// allocator. This entry point serves them; it needs only the distribution
// they already hold and an 8-byte output.
#include <cstdio>
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "../../include/lbm.h"

namespace lbm {
int report_error(int code, const char* msg);
}

namespace {

constexpr int kRowsPerBlock = 8;
constexpr int kThreads = 256;
// One partial per block of kRowsPerBlock rows: up to 32768 rows.
constexpr int kMaxPartials = LBM_NOALLOC_MAX_NY / kRowsPerBlock;

// Shared by every call on a device and kept until the process exits. Each call
// writes every slot it later reads, so nothing has to be cleared first; two
// calls whose kernels overlap on the GPU (different streams, no ordering)
// race on it.
static __device__ __align__(256) double g_partials[kMaxPartials];

// The array's device address is looked up once per device and CUDA context
// (cudaGetSymbolAddress, with that device current) and kept with the context
// it belongs to: a call under another context (a primary context created
// anew after cudaDeviceReset, or a context the caller made current) looks it
// up again instead of using an address of another context.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
    CUcontext ctx;
    double* addr;
};
std::mutex g_mutex;
ScratchAddr g_scratch[kMaxDevices] = {};

// The calling thread's current context, through the driver entry point (the
// library does not link the driver library itself); null if none is current.
CUcontext current_context() {
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    if (fn == nullptr) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || p == nullptr)
            return nullptr;
        fn = (PFN_cuCtxGetCurrent_v4000)p;
    }
    CUcontext c = nullptr;
    return fn(&c) == CUDA_SUCCESS ? c : nullptr;
}

int cuda_error(const char* what, cudaError_t e) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "lbm_total_mass_fp32_noalloc: %s: %s", what, cudaGetErrorString(e));
    return lbm::report_error(LBM_ECUDA, msg);
}

// Block b sums, over the fluid nodes of rows [8b, 8b + 8), rho_ref + the nine
// stored values, in a fixed order (threads stride the rows, then a fixed tree).
__global__ void noalloc_mass_partial(const float* __restrict__ f, int nx, int ny, int pitch,
                                     double rho_ref, const uint8_t* __restrict__ mask,
                                     double* __restrict__ partials) {
    __shared__ double red[kThreads];
    const long long plane = (long long)ny * pitch;
    const int y0 = blockIdx.x * kRowsPerBlock;
    const int y1 = min(y0 + kRowsPerBlock, ny);
    double acc = 0.0;
    for (int y = y0; y < y1; ++y)
        for (int x = threadIdx.x; x < nx; x += kThreads) {
            const long long c = (long long)y * pitch + x;
            if (mask != nullptr && mask[c]) continue;
            double s = rho_ref;
            for (int a = 0; a < 9; ++a) s += (double)f[a * plane + c];
            acc += s;
        }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void noalloc_mass_final(const double* __restrict__ partials, int n, double* out) {
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += partials[b];
    *out = s;
}

}  // namespace

extern "C" int lbm_total_mass_fp32_noalloc(const float* f_dev, int nx, int ny, double rho_ref,
                                           const uint8_t* mask_dev, double* mass_dev,
                                           void* cuda_stream) {
    if (f_dev == nullptr || mass_dev == nullptr)
        return lbm::report_error(LBM_EINVAL, "lbm_total_mass_fp32_noalloc: f_dev and mass_dev must not be null");
    if (nx < 1 || ny < 1)
        return lbm::report_error(LBM_EINVAL, "lbm_total_mass_fp32_noalloc: nx and ny must be >= 1");
    if (ny > LBM_NOALLOC_MAX_NY)
        return lbm::report_error(LBM_EINVAL,
                                 "lbm_total_mass_fp32_noalloc: ny exceeds LBM_NOALLOC_MAX_NY (32768), "
                                 "the capacity of its fixed scratch array");
    const long long pitch = (nx + 31LL) / 32 * 32;
    if (9 * (long long)ny * pitch >= (1LL << 31))
        return lbm::report_error(LBM_EINVAL, "lbm_total_mass_fp32_noalloc: lattice too large (9*ny*pitch >= 2^31)");

    // An error left by earlier asynchronous work is reported as such and left
    // in place (peeked, not cleared), so the caller still sees its own state.
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) return cuda_error("an error from earlier CUDA work is pending", pending);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error("no usable current device", e);
    if (dev < 0 || dev >= kMaxDevices)
        return lbm::report_error(LBM_ECUDA, "lbm_total_mass_fp32_noalloc: device ordinal beyond 63");
    double* partials = nullptr;
    {
        // Set-up once per device and context, with that device current: the
        // host-side name g_partials is not a device address, so ask the
        // runtime for it (this also creates the primary context if none is
        // current yet, hence the context is read again afterwards).
        std::lock_guard<std::mutex> lock(g_mutex);
        CUcontext ctx = current_context();
        if (ctx == nullptr || g_scratch[dev].ctx != ctx || g_scratch[dev].addr == nullptr) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_partials);
            if (e != cudaSuccess || p == nullptr) return cuda_error("cudaGetSymbolAddress failed", e);
            g_scratch[dev] = ScratchAddr{current_context(), (double*)p};
        }
        partials = g_scratch[dev].addr;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int blocks = (ny + kRowsPerBlock - 1) / kRowsPerBlock;
    noalloc_mass_partial<<<blocks, kThreads, 0, s>>>(f_dev, nx, ny, (int)pitch, rho_ref, mask_dev,
                                                     partials);
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_error("partial-sum launch failed", e);
    noalloc_mass_final<<<1, 1, 0, s>>>(partials, blocks, mass_dev);
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) return cuda_error("final-sum launch failed", e);
    return LBM_OK;
}
