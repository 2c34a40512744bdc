// Fused time-step kernel: pull streaming (Eq. 5), density, psi (Eq. 13, 15),
// interaction force (Eq. 7), velocity (Eq. 6), MRT collision with Li's source
// (Eq. 3, 4, 14) and the store of f*, in one pass over HBM.
//
// One CTA updates a TX x TY tile of one lattice of the batch. psi is needed on
// the tile plus a one-node halo; every CTA computes it there itself (pulling
// the nine populations of each halo node, which neighbouring CTAs also read,
// so the extra reads are served by L1/L2) and keeps it in shared memory. Each
// thread keeps its own node's nine pulled populations in registers between the
// psi phase and the collision, so DRAM sees 9 reads + 9 writes per node.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

template <typename T>
struct StepArgs {
    const Tile* tiles;
    const Geom* geom;
    const Phys<T>* phys;
    const T* fin;
    T* fout;
    const uint8_t* mask;
    unsigned* status;
};

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) step_kernel(StepArgs<T> A) {
    constexpr int SW = TX + 2;
    constexpr int SH = TY + 2;
    constexpr int NT = TX * TY;
    constexpr int NH = 2 * SW + 2 * TY;  // halo ring cells
    __shared__ T s_psi[SH * SW];

    const Tile tile = A.tiles[blockIdx.x];
    const Geom g = A.geom[tile.lat];
    const Phys<T>& P = A.phys[tile.lat];
    const T* __restrict__ fin = A.fin + g.f_off;
    const uint8_t* __restrict__ mask = g.has_mask ? A.mask + g.mask_off : nullptr;
    const int plane = (int)g.plane;
    const int nx = g.nx, ny = g.ny, pitch = g.pitch;
    const T rho_ref = P.rho_ref;
    unsigned flag = 0;

    // ---- own node: pull, density, psi
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int x = tile.x0 + lx, y = tile.y0 + ly;
    const bool own = (x < nx) && (y < ny);
    const int xw = own ? x : x % nx;
    const int yw = own ? y : y % ny;
    T f[9];
    const bool solid = pull_node<T>(fin, mask, plane, pitch, nx, ny, xw, yw, f);
    T drho = T(0), rho = T(0), psi = T(-1);
    if (!solid) {
        drho = sum9(f);
        rho = rho_ref + drho;
        if (!(fabs(rho) < T(1e30))) flag |= FLAG_NONFINITE;
        psi = psi_of(rho, P, flag);
    }
    s_psi[(ly + 1) * SW + (lx + 1)] = psi;

    // ---- halo ring: psi only
    for (int h = threadIdx.y * TX + threadIdx.x; h < NH; h += NT) {
        int cx, cy;
        if (h < SW) {
            cx = h;
            cy = 0;
        } else if (h < 2 * SW) {
            cx = h - SW;
            cy = SH - 1;
        } else {
            const int k = h - 2 * SW;
            cy = 1 + (k >> 1);
            cx = (k & 1) ? SW - 1 : 0;
        }
        const int hx = wrap_index(tile.x0 - 1 + cx, nx);
        const int hy = wrap_index(tile.y0 - 1 + cy, ny);
        T fh[9];
        T ph = T(-1);
        if (!pull_node<T>(fin, mask, plane, pitch, nx, ny, hx, hy, fh)) {
            const T rh = rho_ref + sum9(fh);
            ph = psi_of(rh, P, flag);
        }
        s_psi[cy * SW + cx] = ph;
    }
    __syncthreads();

    if (flag) atomicOr(&A.status[tile.lat], flag);
    if (!own || solid) return;

    // ---- force, Eq. 7
    const int c = (ly + 1) * SW + (lx + 1);
    T gx, gy;
    force_sum<T>(psi, s_psi[c + 1], s_psi[c + SW], s_psi[c - 1], s_psi[c - SW],
                 s_psi[c + SW + 1], s_psi[c + SW - 1], s_psi[c - SW - 1], s_psi[c - SW + 1], gx, gy);
    const T mG = -P.G;
    const T Fx = mG * psi * gx;
    const T Fy = mG * psi * gy;
    const T g2G2 = (P.G * P.G) * (gx * gx + gy * gy);

    // ---- collision, Eq. 3
    collide<T>(f, rho, drho, Fx, Fy, g2G2, P);

    // ---- store f*
    T* __restrict__ fo = A.fout + g.f_off + y * pitch + x;
#pragma unroll
    for (int a = 0; a < 9; ++a) fo[a * plane] = f[a];
}

}  // namespace lbm
