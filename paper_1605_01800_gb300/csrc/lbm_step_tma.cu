// TMA-staged, persistent variant of the fused FP32 step kernel.
//
// Same arithmetic per node as step_kernel (lbm_step.cuh), different data
// movement. The tensor maps are __grid_constant__ kernel parameters (per
// lattice: the buffer read this step and the wall mask), so batches of up to
// kTmaMaxLattices lattices can use these variants. Each CTA owns a strided subset of the tile work-list. For a tile
// it needs, per population a, the post-collision values of the tile plus a
// two-cell frame: one 3-D TMA box load per population ({TX+8, TY+4, 1} at
// stored (x0 + kGX - 4, y0 + kGY - 2, a); the x origin is 16-byte aligned) and,
// for a tile within two cells of a solid cell, one 2-D box of the wall mask. The kernel takes the
// tiles at least two cells away from every lattice edge, so a box holds the
// nodes it stands for and no pull wraps; the plain kernel does the others.
// Loads for the next S - 1 tiles are in flight (an mbarrier per stage) while
// the current tile is collided, so the SM has DRAM traffic outstanding
// without holding it in registers. Pulls become shared-memory reads at fixed
// offsets; the CTA's threads store f* to HBM directly (coalesced rows).
//
// Every wait on an mbarrier is bounded (about a second of clock cycles). If a
// stage never completes the CTA records FLAG_TIMEOUT for the lattice, waits
// (bounded again) for the stages it has in flight, and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "lbm_launch.h"
#include "lbm_step.cuh"

namespace lbm {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Spin on the phase with a clock limit; false if it never completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}


// e_a and the opposite population, as compile-time tables for the gathers
__device__ __forceinline__ constexpr int ex_of(int a) {
    return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0);
}
__device__ __forceinline__ constexpr int ey_of(int a) {
    return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0);
}
__device__ __forceinline__ constexpr int opp_of(int a) {
    return a == 0 ? 0 : (a <= 4 ? ((a + 1) & 3) + 1 : ((a - 5 + 2) & 3) + 5);
}

}  // namespace

template <int TX, int TY>
struct TmaBox {
    static constexpr int BW = TX + 8;     // stored x in [x0 - 4, x0 + TX + 4)
    static constexpr int BH = TY + 4;     // stored y in [y0 - 2, y0 + TY + 2)
    static constexpr int BOX = BW * BH;   // floats of one population's box
    static constexpr int BOX_BYTES = BOX * 4;
    static constexpr int MW = TX + 32;    // mask box: x in [x0 - 16, x0 + TX + 16)
    static constexpr int MASK_BYTES = MW * BH;
    static constexpr int STAGE_BYTES = ((9 * BOX_BYTES + MASK_BYTES) + 127) / 128 * 128;
    static_assert(BOX_BYTES % 128 == 0, "population boxes must stay 128-byte aligned");
};

template <int TX, int TY, int RY, int S, int MINB>
__global__ void __launch_bounds__(TX*(TY / RY), MINB)
    step_tma_kernel(const TmaArgs A, const __grid_constant__ TmaMaps M, const __grid_constant__ PhysTable<float> PT) {
    using B = TmaBox<TX, TY>;
    constexpr int TYT = TY / RY;
    constexpr int NT = TX * TYT;
    constexpr int SW = TX + 2;
    constexpr int SH = TY + 2;
    constexpr int NH = 2 * SW + 2 * TY;
    constexpr int NHT = (NH + NT - 1) / NT;
    constexpr int PSI_BYTES = ((SH * SW * 4 + 15) / 16) * 16;
    extern __shared__ __align__(1024) unsigned char smem[];
    // two psi tiles for alternate tiles: a thread may fill the next tile's
    // while others still read this one's, so one barrier per tile suffices
    float* const s_psi2[2] = {reinterpret_cast<float*>(smem + S * B::STAGE_BYTES),
                              reinterpret_cast<float*>(smem + S * B::STAGE_BYTES + PSI_BYTES)};
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * B::STAGE_BYTES + 2 * PSI_BYTES);

    const int tid = threadIdx.y * TX + threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        mbar_init_fence();
    }
    __syncthreads();

    // thread 0: arm stage s for tile t and issue its box loads
    auto issue = [&](int t, int s) {
        const Tile tl = A.tiles[t];
        // a tile with no solid cell within two cells needs no mask box
        const bool has_mask = geom_mask(A.geom[tl.lat]) && !tl.clear;
        unsigned char* st = smem + s * B::STAGE_BYTES;
        mbar_arrive_expect_tx(&bars[s], 9 * B::BOX_BYTES + (has_mask ? B::MASK_BYTES : 0) + A.extra_tx);
        const CUtensorMap* fm = &M.f[tl.lat];
        const int bx = tl.x0 + kGX - 4, by = tl.y0 + kGY - 2;
#pragma unroll
        for (int a = 0; a < 9; ++a) tma_load_3d(st + a * B::BOX_BYTES, fm, bx, by, a, &bars[s]);
        if (has_mask) tma_load_2d(st + 9 * B::BOX_BYTES, &M.m[tl.lat], tl.x0 + kGX - 16, by, &bars[s]);
    };
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            const int t = blockIdx.x + s * gridDim.x;
            if (t < A.n_tiles) issue(t, s);
        }
    }

    int k = 0;
    bool failed = false;
    for (int t = blockIdx.x; t < A.n_tiles; t += gridDim.x, ++k) {
        const int s = k % S;
        const uint32_t parity = (uint32_t)((k / S) & 1);
        // each thread waits for the stage itself; whether every wait
        // succeeded is agreed at the tile's one barrier below (a thread whose
        // wait gave up reads a partial stage there, harmlessly, and stores
        // nothing)
        const bool ok = mbar_wait_bounded(&bars[s], parity, A.wait_limit);
        const Tile tl = A.tiles[t];
        float* const s_psi = s_psi2[k & 1];
        const Geom g = A.geom[tl.lat];
        const Phys<float>* __restrict__ Pp = &PT.p[tl.lat];
        const Phys<float>& P = *Pp;
        const float* __restrict__ st = reinterpret_cast<const float*>(smem + s * B::STAGE_BYTES);
        const uint8_t* __restrict__ ms =
            geom_mask(g) && !tl.clear ? reinterpret_cast<const uint8_t*>(smem + s * B::STAGE_BYTES + 9 * B::BOX_BYTES)
                                      : nullptr;
        const float rho_ref = P.rho_ref;
        unsigned flag = 0;

        // pulled populations of the cell at tile-local (lx, ly), lx in [-1, TX],
        // ly in [-1, TY]; false if the cell is solid
        auto gather = [&](int lx, int ly, float f[9]) -> bool {
            const int o = (ly + 2) * B::BW + (lx + 4);  // the cell itself in every box
            if (ms != nullptr) {
                const int mo = (ly + 2) * B::MW + (lx + 16);
                if (ms[mo]) return false;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const int d = ey_of(a) * B::BW + ex_of(a);
                    const int md = ey_of(a) * B::MW + ex_of(a);
                    f[a] = (a != 0 && ms[mo - md]) ? st[opp_of(a) * B::BOX + o] : st[a * B::BOX + o - d];
                }
                return true;
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) f[a] = st[a * B::BOX + o - (ey_of(a) * B::BW + ex_of(a))];
            return true;
        };

        // ---- own nodes
        float f[RY][9];
        bool live[RY];
        float drho[RY], rho[RY], psi[RY];
        const int lx = threadIdx.x;
        const int x = tl.x0 + lx;
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int ly = threadIdx.y * RY + r;
            const int y = tl.y0 + ly;
            live[r] = (x <= g.nx) && (y <= g.ny);
            if (live[r]) live[r] = gather(lx, ly, f[r]);
        }
        f32_rho_psi<RY>(f, live, rho_ref, P, flag, drho, rho, psi);
#pragma unroll
        for (int r = 0; r < RY; ++r) s_psi[(threadIdx.y * RY + r + 1) * SW + (lx + 1)] = psi[r];
        // ---- halo ring: psi only
#pragma unroll
        for (int j = 0; j < NHT; ++j) {
            const int h = tid + j * NT;
            if (h < NH) {
                int cx, cy;
                if (h < SW) {
                    cx = h;
                    cy = 0;
                } else if (h < 2 * SW) {
                    cx = h - SW;
                    cy = SH - 1;
                } else {
                    const int q = h - 2 * SW;
                    cy = 1 + (q >> 1);
                    cx = (q & 1) ? SW - 1 : 0;
                }
                float ph = -1.0f;
                float fh[9];
                if (tl.x0 - 1 + cx <= g.nx && tl.y0 - 1 + cy <= g.ny && gather(cx - 1, cy - 1, fh))
                    ph = f32_halo_psi(fh, rho_ref, P, flag);
                s_psi[cy * SW + cx] = ph;
            }
        }
        // stage s consumed, psi tile complete; and every wait succeeded
        if (__syncthreads_or(!ok)) {
            failed = true;
            if (tid == 0) atomicOr(&A.status[tl.lat], FLAG_TIMEOUT);
            break;
        }

        if (tid == 0) {
            const int tn = t + S * gridDim.x;
            if (tn < A.n_tiles) {
                fence_proxy_async();  // generic reads of stage s before the async refill
                issue(tn, s);
            }
        }
        if (flag) atomicOr(&A.status[tl.lat], flag);

        if (x < g.nx)
            f32_collide_store<RY, SW>(f, live, drho, rho, psi, s_psi, lx, threadIdx.y * RY, ms != nullptr, P,
                                      A.fout + g.f_off, g, x, tl.y0 + threadIdx.y * RY);
        // this psi tile is written again two tiles on, after the next
        // tile's barrier, which every thread reaches after this collision
    }

    if (failed && tid == 0) {
        // wait (bounded) for the loads still in flight into this CTA's stages;
        // copies land within microseconds, so 50 ms is ample even when the
        // waits above were shortened
        const long long drain = A.wait_limit > 100000000LL ? A.wait_limit : 100000000LL;
        for (int j = 0; j < S; ++j) {
            const int kk = k + j;
            const int t = blockIdx.x + kk * gridDim.x;
            if (t < A.n_tiles) mbar_wait_bounded(&bars[kk % S], (uint32_t)((kk / S) & 1), drain);
        }
    }
}

// ---------------------------------------------------------------- host side

template <int TX, int TY, int RY, int S>
constexpr size_t tma_smem_bytes() {
    using B = TmaBox<TX, TY>;
    return (size_t)S * B::STAGE_BYTES + 2 * (((TX + 2) * (TY + 2) * 4 + 15) / 16) * 16 + S * sizeof(uint64_t);
}

template <int TX, int TY, int RY, int S, int MINB>
static cudaError_t launch_tma_tile(int grid, const TmaArgs& a, const TmaMaps& maps, const PhysTable<float>& table,
                                   cudaStream_t s) {
    const size_t smem = tma_smem_bytes<TX, TY, RY, S>();
    static bool configured = false;  // per process; attributes are per device but identical
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(step_tma_kernel<TX, TY, RY, S, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    step_tma_kernel<TX, TY, RY, S, MINB><<<grid, dim3(TX, TY / RY), smem, s>>>(a, maps, table);
    return cudaGetLastError();
}

template <int TX, int TY, int RY, int S, int MINB>
static int tma_occupancy() {
    const size_t smem = tma_smem_bytes<TX, TY, RY, S>();
    if (cudaFuncSetAttribute(step_tma_kernel<TX, TY, RY, S, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_tma_kernel<TX, TY, RY, S, MINB>, TX * (TY / RY), smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// TMA variants: {TX, TY, RY, stages, minimum resident CTAs per SM (the
// register cap)}
#define LBM_TMA_VARIANTS(X) X(0, 32, 8, 1, 3, 3) X(1, 32, 16, 2, 2, 3) X(2, 32, 16, 2, 2, 4) X(3, 32, 16, 2, 3, 2)

int tma_variant_count() { return 4; }

void tma_variant_shape(int v, int* tx, int* ty) {
#define LBM_SHAPE(i, a, b, r, s, m) \
    if (v == i) {                \
        *tx = a;                 \
        *ty = b;                 \
    }
    LBM_TMA_VARIANTS(LBM_SHAPE)
#undef LBM_SHAPE
}

int tma_plain_partner(int v) {
    int tx = 0, ty = 0;
    tma_variant_shape(v, &tx, &ty);
    for (int i = 0; i < kTileCount; ++i)
        if (kTiles[i][0] == tx && kTiles[i][1] * kTiles[i][2] == ty) return i;
    return -1;
}

int tma_blocks_per_sm(int v) {
#define LBM_OCC(i, a, b, r, s, m) \
    if (v == i) return tma_occupancy<a, b, r, s, m>();
    LBM_TMA_VARIANTS(LBM_OCC)
#undef LBM_OCC
    return 0;
}

cudaError_t launch_step_tma(int v, int grid, const TmaArgs& args, const TmaMaps& maps,
                            const PhysTable<float>& table, cudaStream_t s) {
    if (args.n_tiles <= 0) return cudaSuccess;
#define LBM_LAUNCH(i, a, b, r, st, m) \
    if (v == i) return launch_tma_tile<a, b, r, st, m>(grid, args, maps, table, s);
    LBM_TMA_VARIANTS(LBM_LAUNCH)
#undef LBM_LAUNCH
    return cudaErrorInvalidValue;
}

// Tensor maps of one lattice's planes in a distribution buffer (3-D: x, y,
// population) and of its wall mask (2-D), boxes sized for tile TX x TY.
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn == nullptr) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

bool encode_lattice_maps(const Geom& g, int tx, int ty, const float* buf0, const float* buf1,
                         const uint8_t* mask_base, CUtensorMap* fmaps2, CUtensorMap* mmap) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (enc == nullptr) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.ny + 2 * kGY), 9};
    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4};
    const cuuint32_t box[3] = {(cuuint32_t)(tx + 8), (cuuint32_t)(ty + 4), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const float* bufs[2] = {buf0, buf1};
    for (int b = 0; b < 2; ++b) {
        CUresult r = enc(&fmaps2[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)(bufs[b] + g.f_off), dims, strides,
                         box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    if (geom_mask(g)) {
        const cuuint64_t mdims[2] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.ny + 2 * kGY)};
        const cuuint64_t mstr[1] = {(cuuint64_t)g.pitch};
        const cuuint32_t mbox[2] = {(cuuint32_t)(tx + 32), (cuuint32_t)(ty + 4)};
        const cuuint32_t mestr[2] = {1, 1};
        CUresult r = enc(mmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)(mask_base + g.mask_off), mdims, mstr, mbox,
                         mestr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    } else {
        memset(mmap, 0, sizeof(CUtensorMap));
    }
    return true;
}

}  // namespace lbm
