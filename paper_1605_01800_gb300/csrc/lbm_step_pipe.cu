// Persistent, software-pipelined FP32 step kernel for full wall-free tiles.
//
// Same arithmetic per node as the fast path of step_kernel (lbm_step.cuh),
// different scheduling. The plain kernel runs one CTA per tile, and a CTA's
// loads, its psi exchange and its collision run in sequence, so on a batch of
// a few waves the SMs alternate between waiting on DRAM and computing. Here
// each CTA walks the list of fast tiles with a stride of the grid size and
// keeps two register sets: after the psi barrier of tile k it issues the
// pulled loads of its next tile (own node pairs and its halo cell) and only
// then does the force, the collision and the stores of tile k, so those loads
// are in flight while it computes. Tiles within two cells of a lattice edge
// wrap the pulls that cross it, as in step_kernel's fast path. Tiles that
// need the general path (partial tiles, walls, lattices under 4 x 4) go
// through step_kernel in a second launch of the same step; the two launches
// write disjoint nodes.
#include "lbm_launch.h"
#include "lbm_step.cuh"

namespace lbm {

namespace {

// pulled populations of a thread's node pair and of its halo cell (if any)
__device__ __forceinline__ void pipe_load(const float* __restrict__ fin, const FastTile& T, int lx, int ly0,
                                          bool has_h, int hcx, int hcy, F2 f[9], float fh[9]) {
    const float* __restrict__ base = fin + T.f_off;
    const int pitch = T.pitch, plane = T.plane;
    const int x = T.x0 + lx, y = T.y0 + ly0;
    const int c = (y + kGY) * pitch + x + kGX;
    const int hx = T.x0 - 1 + hcx, hy = T.y0 - 1 + hcy;
    if (T.edge) {
        const int dxm = x == 0 ? T.nx - 1 : -1;
        const int dxp = x == T.nx - 1 ? 1 - T.nx : 1;
        const int rm = y == 0 ? (T.ny - 1) * pitch : -pitch;
        const int rp2 = y + 1 == T.ny - 1 ? (1 - T.ny) * pitch : pitch;
        pull_pair_wrap(base, plane, pitch, c, dxm, dxp, rm, rp2, f);
        if (has_h) pull_node<float>(base, nullptr, plane, nbr_of(T.nx, T.ny, pitch, hx, hy), fh);
    } else {
        pull_pair(base, plane, pitch, c, f);
        if (has_h) pull_inner<float>(base, plane, pitch, (hy + kGY) * pitch + hx + kGX, fh);
    }
}

template <int TX, int TYT, int MINB, bool TABLE>
__global__ void __launch_bounds__(TX * TYT, MINB)
    step_pipe_kernel(const PipeArgs A, const __grid_constant__ TableOf<float, TABLE> PT) {
    constexpr int TY = 2 * TYT;
    constexpr int SW = TX + 2;
    constexpr int SH = TY + 2;
    constexpr int NT = TX * TYT;
    constexpr int NH = 2 * SW + 2 * TY;
    static_assert(NH <= NT, "one halo cell per thread at most");
    __shared__ float s_psi[SH * SW];

    const int lx = threadIdx.x, ly0 = 2 * threadIdx.y;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const bool has_h = tid < NH;
    int hcx = 0, hcy = 0;
    if (has_h) halo_ring_cell<SW, SH>(tid, hcx, hcy);
    const int hc = hcy * SW + hcx;

    int t = blockIdx.x;
    if (t >= A.n_fast) return;
    FastTile T = A.fast[t];
    F2 f[9];
    float fh[9];
    pipe_load(A.fin, T, lx, ly0, has_h, hcx, hcy, f, fh);
    for (;;) {
        const int tn = t + (int)gridDim.x;
        const bool more = tn < A.n_fast;
        FastTile Tn;
        if (more) Tn = A.fast[tn];
#ifdef LBM_DEBUG
        // debug builds poison the psi tile of every tile (see step_kernel)
        for (int i = tid; i < SH * SW; i += NT) s_psi[i] = NAN;
        __syncthreads();
#endif
        const Phys<float>* __restrict__ Pp;
        if constexpr (TABLE)
            Pp = &PT.p[T.lat];
        else
            Pp = A.phys + T.lat;
        const Phys<float>& P = *Pp;
        const float rho_ref = P.rho_ref;
        unsigned flag = 0;

        // density and psi of the node pair and of the halo cell
        const F2 drho = vsum9(f);
        const F2 rho = splat<F2>(rho_ref) + drho;
        const F2 psi = vpsi(rho, P, flag);
        s_psi[(ly0 + 1) * SW + lx + 1] = psi.v.x;
        s_psi[(ly0 + 2) * SW + lx + 1] = psi.v.y;
        if (has_h) s_psi[hc] = f32_halo_psi<false>(fh, rho_ref, P, flag);
        __syncthreads();
        if (flag) atomicOr(&A.status[T.lat], flag);

        // the next tile's loads go out before this tile's collision
        F2 fn[9];
        float fhn[9];
        if (more) pipe_load(A.fin, Tn, lx, ly0, has_h, hcx, hcy, fn, fhn);

        const int x = T.x0 + lx, y = T.y0 + ly0;
        f32_pair_finish<SW>(f, rho, drho, psi, s_psi, lx, ly0, P, A.fout + T.f_off,
                            (y + kGY) * T.pitch + x + kGX, T.plane, T.pitch);
        __syncthreads();  // s_psi is rewritten by the next tile
        if (!more) break;
        t = tn;
        T = Tn;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            f[a] = fn[a];
            fh[a] = fhn[a];
        }
    }
}

// Pipelined shapes {TX, TYT, MINB}; the node tile is TX x 2 TYT.
constexpr int kPipeShapes[][3] = {{32, 4, 4}, {32, 8, 2}, {64, 4, 2}};
constexpr int kPipeCount = sizeof(kPipeShapes) / sizeof(kPipeShapes[0]);

template <int TX, int TYT, int MINB>
int pipe_blocks_per_sm(bool table) {
    int n = 0;
    cudaError_t e = table ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                &n, step_pipe_kernel<TX, TYT, MINB, true>, TX * TYT, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                &n, step_pipe_kernel<TX, TYT, MINB, false>, TX * TYT, 0);
    return e == cudaSuccess ? n : 0;
}

template <int TX, int TYT, int MINB>
cudaError_t launch_pipe(int grid, const PipeArgs& a, const PhysTable<float>* table, cudaStream_t s) {
    if (table) {
        step_pipe_kernel<TX, TYT, MINB, true><<<grid, dim3(TX, TYT), 0, s>>>(a, *table);
    } else {
        step_pipe_kernel<TX, TYT, MINB, false><<<grid, dim3(TX, TYT), 0, s>>>(a, NoTable{0});
    }
    return cudaGetLastError();
}

}  // namespace

int pipe_variant_count() { return kPipeCount; }

void pipe_variant_shape(int v, int* tx, int* ty) {
    *tx = kPipeShapes[v][0];
    *ty = 2 * kPipeShapes[v][1];
}

// plain step_kernel shape (index into kTiles) with the same node tile, for
// the tiles the pipelined kernel does not take
int pipe_plain_partner(int v) {
    for (int i = 0; i < kTileCount; ++i)
        if (kTiles[i][0] == kPipeShapes[v][0] && kTiles[i][1] * kTiles[i][2] == 2 * kPipeShapes[v][1] &&
            kTiles[i][2] == 2)
            return i;
    return -1;
}

#define LBM_PIPE_CASES(X) X(0, 32, 4, 4) X(1, 32, 8, 2) X(2, 64, 4, 2)

int pipe_blocks_per_sm(int v, bool table) {
    switch (v) {
#define X(i, tx, tyt, minb) \
    case i: return pipe_blocks_per_sm<tx, tyt, minb>(table);
        LBM_PIPE_CASES(X)
#undef X
    default: return 0;
    }
}

cudaError_t launch_step_pipe(int v, int grid, const PipeArgs& a, const PhysTable<float>* table, cudaStream_t s) {
    if (a.n_fast <= 0 || grid <= 0) return cudaSuccess;
    switch (v) {
#define X(i, tx, tyt, minb) \
    case i: return launch_pipe<tx, tyt, minb>(grid, a, table, s);
        LBM_PIPE_CASES(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
