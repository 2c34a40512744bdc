// Fused time-step kernel: pull streaming (Eq. 5), density, psi (Eq. 13, 15),
// interaction force (Eq. 7), velocity (Eq. 6), MRT collision with Li's source
// (Eq. 3, 4, 14) and the store of f*, in one pass over HBM.
//
// One CTA of TX x TYT threads updates a TX x (TYT * RY) tile of one lattice of
// the batch; each thread owns RY vertically adjacent nodes of one column. psi
// is needed on the tile plus a one-node halo: the CTA computes it there itself
// (pulling the nine populations of each halo node, which neighbouring CTAs
// also read, so those reads hit L2) and keeps it in shared memory. Each
// thread's own nodes keep their nine pulled populations in registers between
// the psi phase and the collision, so DRAM sees 9 reads + 9 writes per node
// (plus the ghost images of edge nodes). The ghost frame of the layout makes
// every pull a fixed offset. All RY * 9 loads of a thread are issued before
// any of them is used.
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

// Register cap for the FP32 kernel with up to two nodes per thread: 64 per
// thread, so that 1024 threads per SM are resident.
template <typename T, int TX, int TYT, int RY>
__global__ void __launch_bounds__(TX * TYT, (sizeof(T) == 4 && RY <= 2) ? 1024 / (TX * TYT) : 1)
    step_kernel(StepArgs<T> A) {
    constexpr int TY = TYT * RY;
    constexpr int SW = TX + 2;
    constexpr int SH = TY + 2;
    constexpr int NT = TX * TYT;
    constexpr int NH = 2 * SW + 2 * TY;  // halo ring cells
    __shared__ T s_psi[SH * SW];

    const Tile tile = A.tiles[blockIdx.x];
    const Geom g = A.geom[tile.lat];
    // restrict: the stores to fout cannot alias the parameters, so they need
    // not be reloaded after every store
    const Phys<T>* __restrict__ Pp = A.phys + tile.lat;
    const Phys<T>& P = *Pp;
    const T* __restrict__ fin = A.fin + g.f_off;
    const uint8_t* __restrict__ mask = g.has_mask ? A.mask + g.mask_off : nullptr;
    const int plane = (int)g.plane;
    const int nx = g.nx, ny = g.ny, pitch = g.pitch;
    const T rho_ref = P.rho_ref;
    unsigned flag = 0;

    // ---- own nodes: column x, rows y0 .. y0 + RY - 1. Cells past the last
    // node (a tile overhanging the lattice) are pulled only up to x = nx and
    // y = ny, the ghost images the last nodes' forces need.
    const int lx = threadIdx.x;
    const int x = tile.x0 + lx;
    const int y0 = tile.y0 + threadIdx.y * RY;
    T f[RY][9];
    bool live[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int y = y0 + r;
        live[r] = (x <= nx) && (y <= ny);
        if (live[r]) live[r] = !pull_node<T>(fin, mask, plane, pitch, node_index(g, x, y), f[r]);
    }

    // ---- halo ring: psi only (issued before the own nodes' arithmetic)
    T ph[(NH + NT - 1) / NT];
    int hc[(NH + NT - 1) / NT];
    const int tid = threadIdx.y * TX + threadIdx.x;
#pragma unroll
    for (int k = 0; k < (NH + NT - 1) / NT; ++k) {
        const int h = tid + k * NT;
        hc[k] = -1;
        ph[k] = T(-1);
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
            hc[k] = cy * SW + cx;
            const int hx = tile.x0 - 1 + cx, hy = tile.y0 - 1 + cy;
            T fh[9];
            if (hx <= nx && hy <= ny &&
                !pull_node<T>(fin, mask, plane, pitch, node_index(g, hx, hy), fh)) {
                const T rh = rho_ref + sum9(fh);
                ph[k] = psi_of(rh, P, flag);
            }
        }
    }

    // ---- own nodes: density and psi
    T drho[RY], rho[RY], psi[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        drho[r] = T(0);
        rho[r] = T(0);
        psi[r] = T(-1);
        if (live[r]) {
            drho[r] = sum9(f[r]);
            rho[r] = rho_ref + drho[r];
            psi[r] = psi_of(rho[r], P, flag);
        }
        s_psi[(threadIdx.y * RY + r + 1) * SW + (lx + 1)] = psi[r];
    }
#pragma unroll
    for (int k = 0; k < (NH + NT - 1) / NT; ++k)
        if (hc[k] >= 0) s_psi[hc[k]] = ph[k];
    __syncthreads();

    if (flag) atomicOr(&A.status[tile.lat], flag);
    if (x >= nx) return;

    const T mG = -P.G;
    const T G2 = P.G * P.G;
    T* __restrict__ fo = A.fout + g.f_off;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int y = y0 + r;
        if (y >= ny || !live[r]) continue;
        // ---- force, Eq. 7
        const int c = (threadIdx.y * RY + r + 1) * SW + (lx + 1);
        T gx, gy;
        force_sum<T>(mask != nullptr, psi[r], s_psi[c + 1], s_psi[c + SW], s_psi[c - 1], s_psi[c - SW],
                     s_psi[c + SW + 1], s_psi[c + SW - 1], s_psi[c - SW - 1], s_psi[c - SW + 1], gx,
                     gy);
        const T Fx = mG * psi[r] * gx;
        const T Fy = mG * psi[r] * gy;
        // ---- collision, Eq. 3
        collide<T>(f[r], rho[r], drho[r], Fx, Fy, G2 * (gx * gx + gy * gy), P);
        // ---- store f* (and its ghost images near an edge)
        store_node<T>(fo, g, x, y, f[r]);
    }
}

}  // namespace lbm
