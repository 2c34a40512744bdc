// Time step of in-place storage (one distribution array, the AA pattern; the
// two layouts are described at kLayoutPull in lbm_device.cuh).
//
// The fused two-buffer kernel recomputes psi on a one-node ring around its
// tile from the neighbours' populations. In place, those populations are
// overwritten by the neighbouring CTAs during the same launch, so psi comes
// from a pass of its own: launch 1 gathers every node's distribution,
// computes rho and psi (Eq. 13, 15) and writes psi to a plane with a
// one-cell periodic frame (-1 at solid nodes); launch 2 gathers the
// distribution again, reads the node's and its eight neighbours' psi from
// the plane, and applies the force (Eq. 7), the collision (Eq. 3, 4, 14) and
// the store in the other layout. Per node and step: 36 + 4 bytes for launch
// 1, 36 + 4 + 36 for launch 2 (the neighbours' psi come from L1/L2), against
// 72 for the two-buffer step; the distribution takes 36 bytes per node
// instead of 72.
//
// The arithmetic is that of the two-buffer kernel operation for operation
// (the FP32 node functions of lbm_device.cuh one node at a time, the FP64
// ones of its general path), so both storages give bitwise the same fields.
#include "lbm_launch.h"

namespace lbm {

namespace {

// rho - rho_ref and rho of a gathered node, and its psi, as the two-buffer
// kernel computes them
__device__ __forceinline__ void node_rho(const float (&f)[9], float rho_ref, float& drho, float& rho) {
    F1 v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a].v = f[a];
    const F1 d = vsum9(v);
    drho = d.v;
    rho = (splat<F1>(rho_ref) + d).v;
}
__device__ __forceinline__ void node_rho(const double (&f)[9], double rho_ref, double& drho, double& rho) {
    drho = sum9(f);
    rho = rho_ref + drho;
}
__device__ __forceinline__ float node_psi(float rho, const Phys<float>& P, unsigned& flag) {
    return vpsi_any(F1{rho}, P, flag).v;
}
__device__ __forceinline__ double node_psi(double rho, const Phys<double>& P, unsigned& flag) {
    return psi_of(rho, P, flag);
}

// force (Eq. 7) and collision of one fluid node from its psi and its eight
// neighbours' (nb: E, N, W, S, NE, NW, SW, SE; a negative entry is a solid
// neighbour, which takes the node's psi on lattices with walls)
__device__ __forceinline__ void node_collide(float (&f)[9], float rho, float drho, float psi, float (&nb)[8],
                                             bool walls, const Phys<float>& P) {
    if (walls) {
#pragma unroll
        for (int k = 0; k < 8; ++k) nb[k] = nb[k] < 0.0f ? psi : nb[k];
    }
    F1 n[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) n[k].v = nb[k];
    F1 gx, gy;
    vforce_sum(n[0], n[1], n[2], n[3], n[4], n[5], n[6], n[7], gx, gy);
    const F1 mGpsi = splat<F1>(-P.G) * F1{psi};
    const F1 Fx = mGpsi * gx, Fy = mGpsi * gy;
    const F1 g2G2 = splat<F1>(__fmul_rn(P.G, P.G)) * vfma(gx, gx, gy * gy);
    F1 v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a].v = f[a];
    vcollide(v, F1{rho}, F1{drho}, Fx, Fy, g2G2, P);
#pragma unroll
    for (int a = 0; a < 9; ++a) f[a] = v[a].v;
}
__device__ __forceinline__ void node_collide(double (&f)[9], double rho, double drho, double psi, double (&nb)[8],
                                             bool walls, const Phys<double>& P) {
    const double mG = -P.G;
    const double G2 = P.G * P.G;
    double gx, gy;
    force_sum<double>(walls, psi, nb[0], nb[1], nb[2], nb[3], nb[4], nb[5], nb[6], nb[7], gx, gy);
    const double Fx = mG * psi * gx;
    const double Fy = mG * psi * gy;
    collide<double>(f, rho, drho, Fx, Fy, G2 * (gx * gx + gy * gy), P);
}

// A CTA of kIpThreads threads walks its tile's nodes in NPT rounds: node
// q = j * kIpThreads + tid (j < NPT) in row-major order of the tile; every
// thread issues the loads of all its nodes before it computes any of them.
// NPT = tile nodes / kIpThreads.
constexpr int kIpThreads = 128;

__device__ __forceinline__ bool ip_node(const Tile& tile, const Geom& g, int tx, int j, int& x, int& y) {
    const int q = j * kIpThreads + (int)threadIdx.x;
    const int ly = q / tx, lx = q - ly * tx;
    x = tile.x0 + lx;
    y = tile.y0 + ly;
    return x < g.nx && y < g.ny;
}

// Launch 1: psi of every node of the CTA's tile into the plane, and into the
// frame cells that stand for it across the lattice's edges.
template <typename T, int LAYOUT, int NPT>
__global__ void __launch_bounds__(kIpThreads)
    inplace_psi_kernel(const TileGeom* __restrict__ tg, int tx, const Phys<T>* __restrict__ phys,
                       const T* __restrict__ f_base, const uint8_t* __restrict__ mask_base, T* __restrict__ psi_base,
                       unsigned* __restrict__ status) {
    const Tile tile = tg[blockIdx.x].t;
    const Geom g = tg[blockIdx.x].g;
    const Phys<T>& P = phys[tile.lat];
    // no solid cell within two cells of a clear tile: no mask lookups
    const uint8_t* mask = geom_mask(g) && !tile.clear ? mask_base + g.mask_off : nullptr;
    const T* f = f_base + g.f_off;
    T* psi = psi_base + g.f_off / 9;
    const int plane = (int)g.plane;
    T fv[NPT][9];
    bool live[NPT], solid[NPT];
    int xj[NPT], yj[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        live[j] = ip_node(tile, g, tx, j, xj[j], yj[j]);
        solid[j] = true;
        if (live[j]) solid[j] = gather_node<T>(LAYOUT, f, mask, plane, nbr_of(g.nx, g.ny, g.pitch, xj[j], yj[j]), fv[j]);
    }
    unsigned flag = 0;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        if (!live[j]) continue;
        const int x = xj[j], y = yj[j];
        T ps = T(-1);
        if (!solid[j]) {
            T drho, rho;
            node_rho(fv[j], P.rho_ref, drho, rho);
            ps = node_psi(rho, P, flag);
        }
        // the node and its periodic images in the one-cell frame
        // (x = -1, nx; y = -1, ny), three each way on a lattice one node
        // wide or high
        int xs[3], ys[3], kx = 0, ky = 0;
        xs[kx++] = x;
        if (x == 0) xs[kx++] = g.nx;
        if (x == g.nx - 1) xs[kx++] = -1;
        ys[ky++] = y;
        if (y == 0) ys[ky++] = g.ny;
        if (y == g.ny - 1) ys[ky++] = -1;
        for (int b = 0; b < ky; ++b)
            for (int a = 0; a < kx; ++a) psi[node_index(g, xs[a], ys[b])] = ps;
    }
    if (flag) atomicOr(&status[tile.lat], flag);
}

// Launch 2: force, collision and the store of every fluid node of the CTA's
// tile, from the distribution in LAYOUT into the other layout.
template <typename T, int LAYOUT, int NPT>
__global__ void __launch_bounds__(kIpThreads)
    inplace_collide_kernel(const TileGeom* __restrict__ tg, int tx, const Phys<T>* __restrict__ phys,
                           T* __restrict__ f_base, const uint8_t* __restrict__ mask_base,
                           const T* __restrict__ psi_base) {
    const Tile tile = tg[blockIdx.x].t;
    const Geom g = tg[blockIdx.x].g;
    const Phys<T>& P = phys[tile.lat];
    // no solid cell within two cells of a clear tile: no mask lookups
    const uint8_t* mask = geom_mask(g) && !tile.clear ? mask_base + g.mask_off : nullptr;
    T* f = f_base + g.f_off;
    const T* psi = psi_base + g.f_off / 9;
    const int plane = (int)g.plane, pitch = g.pitch, np = 9 * plane;
    T fv[NPT][9];
    bool go[NPT];
    int xj[NPT], yj[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        go[j] = ip_node(tile, g, tx, j, xj[j], yj[j]);
        if (go[j]) go[j] = !gather_node<T>(LAYOUT, f, mask, plane, nbr_of(g.nx, g.ny, pitch, xj[j], yj[j]), fv[j]);
    }
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        if (!go[j]) continue;
        const Nbr n = nbr_of(g.nx, g.ny, pitch, xj[j], yj[j]);
        // rho as the psi pass computed it (same operations); psi from the
        // plane (the pass's value)
        T drho, rho;
        node_rho(fv[j], P.rho_ref, drho, rho);
        const int c = n.c;
        const T own = psi[c];
        T nb[8] = {psi[c + 1],         psi[c + pitch],     psi[c - 1],         psi[c - pitch],
                   psi[c + pitch + 1], psi[c + pitch - 1], psi[c - pitch - 1], psi[c - pitch + 1]};
        node_collide(fv[j], rho, drho, own, nb, mask != nullptr, P);
        if (LAYOUT == kLayoutNatural) {
            // collided in place: f*_a to plane opp(a) of the node
#pragma unroll
            for (int a = 0; a < 9; ++a) st_pop<T>(f, opp(a) * plane + c, np, fv[j][a]);
        } else {
            // streamed: f*_a to plane a of x + e_a, or back to plane opp(a)
            // of the node when x + e_a is solid
            st_pop<T>(f, c, np, fv[j][0]);
#pragma unroll
            for (int a = 1; a < 9; ++a) {
                const int t = c + nbr_offset(n, a);
                if (mask != nullptr && ld_mask(mask, t, plane))
                    st_pop<T>(f, opp(a) * plane + c, np, fv[j][a]);
                else
                    st_pop<T>(f, a * plane + t, np, fv[j][a]);
            }
        }
    }
}

template <typename T, int LAYOUT, int NPT>
cudaError_t step_layout(const TileGeom* tg, int n_tiles, int tx, const Phys<T>* phys, T* f, const uint8_t* mask,
                        T* psi, unsigned* status, cudaStream_t s) {
    inplace_psi_kernel<T, LAYOUT, NPT><<<n_tiles, kIpThreads, 0, s>>>(tg, tx, phys, f, mask, psi, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    inplace_collide_kernel<T, LAYOUT, NPT><<<n_tiles, kIpThreads, 0, s>>>(tg, tx, phys, f, mask, psi);
    return cudaGetLastError();
}

template <typename T, int NPT>
cudaError_t step_npt(const TileGeom* tg, int n_tiles, int tx, const Phys<T>* phys, T* f, const uint8_t* mask,
                     T* psi, unsigned* status, int layout, cudaStream_t s) {
    return layout == kLayoutNatural
               ? step_layout<T, kLayoutNatural, NPT>(tg, n_tiles, tx, phys, f, mask, psi, status, s)
               : step_layout<T, kLayoutSwapped, NPT>(tg, n_tiles, tx, phys, f, mask, psi, status, s);
}

template <typename T>
cudaError_t step_inplace(const TileGeom* tg, int n_tiles, int tx, int ty, const Phys<T>* phys, T* f,
                         const uint8_t* mask, T* psi, unsigned* status, int layout, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    switch (tx * ty) {
        case 2 * kIpThreads: return step_npt<T, 2>(tg, n_tiles, tx, phys, f, mask, psi, status, layout, s);
        case 4 * kIpThreads: return step_npt<T, 4>(tg, n_tiles, tx, phys, f, mask, psi, status, layout, s);
        default: return cudaErrorInvalidValue;  // every built-in plain tile holds 256 or 512 nodes
    }
}

}  // namespace

cudaError_t launch_step_inplace_f32(const TileGeom* tg, int n_tiles, int tx, int ty, const Phys<float>* phys,
                                    float* f, const uint8_t* mask, float* psi, unsigned* status, int layout,
                                    cudaStream_t s) {
    return step_inplace<float>(tg, n_tiles, tx, ty, phys, f, mask, psi, status, layout, s);
}
cudaError_t launch_step_inplace_f64(const TileGeom* tg, int n_tiles, int tx, int ty, const Phys<double>* phys,
                                    double* f, const uint8_t* mask, double* psi, unsigned* status, int layout,
                                    cudaStream_t s) {
    return step_inplace<double>(tg, n_tiles, tx, ty, phys, f, mask, psi, status, layout, s);
}

}  // namespace lbm
