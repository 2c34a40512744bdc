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
// the psi phase and the collision, so DRAM sees 9 reads + 9 writes per node.
// Pulls inside a lattice are fixed offsets; tiles at a lattice edge wrap the
// pulls that cross it (nbr_of). All RY * 9 loads of a thread are issued
// before any of them is used.
#pragma once

#include <type_traits>

#include "lbm_device.cuh"

namespace lbm {

// Per-lattice parameters as a kernel parameter (constant bank): indexed by
// the CTA's lattice, a warp-uniform value, they load once into uniform
// registers instead of being re-read from global memory under register
// pressure. Used when a batch has at most kParamLattices lattices.
constexpr int kParamLattices = 64;
template <typename T>
struct PhysTable {
    Phys<T> p[kParamLattices];
};
struct NoTable {
    int unused;
};
template <typename T, bool TABLE>
using TableOf = typename std::conditional<TABLE, PhysTable<T>, NoTable>::type;

// A work-list that is a regular grid of tiles (see tile_at): tiles_x tiles
// per row of a lattice, tiles_per_lat per lattice, lattice l's populations
// at g0.f_off + l * lat_stride. tiles_x == 0: not a grid. The divisions by
// tiles_per_lat and tiles_x are a multiplication and a shift (div_magic).
struct TileGrid {
    int tiles_x, tiles_per_lat;
    long long lat_stride;
    Geom g0;
    unsigned long long m_lat, m_x;  // magic multipliers of tiles_per_lat and tiles_x
    int s_lat, s_x;                 // their shifts
};

// Division by a constant d as a multiplication and a shift (Granlund and
// Montgomery's method, "Division by invariant integers using
// multiplication", 1994): with s = ceil(log2 d) and m = ceil(2^(32+s) / d),
// floor(n / d) = (n m) >> (32 + s) for every 0 <= n < 2^31 (the error of m,
// below 1/d per unit of 2^(32+s), adds less than 1/(2d) to n/d), and n m
// stays below 2^64.
inline void div_magic_of(int d, unsigned long long* m, int* s) {
    int l = 0;
    while ((1ll << l) < (long long)d) ++l;
    *s = l;
    *m = ((1ull << (32 + l)) + (unsigned long long)d - 1) / (unsigned long long)d;
}
__device__ __forceinline__ int div_magic(int n, unsigned long long m, int s) {
    return (int)(((unsigned long long)(unsigned)n * m) >> (32 + s));
}

template <typename T>
struct StepArgs {
    const Tile* tiles;
    const Geom* geom;
    const Phys<T>* phys;
    const T* fin;
    T* fout;
    const uint8_t* mask;
    unsigned* status;
    const TileGeom* tg;  // per entry of `tiles`: the tile and its lattice's geometry
    // L2 prefetch distance in CTAs (0: none). The callers of the launch
    // functions pass 1 (prefetch) or 0; the launch functions set the distance.
    int ahead;
};

// The list as a regular grid of tiles (G.tiles_x > 0, a kernel argument of
// its own after the others): every lattice of the batch has the geometry
// G.g0 (its f_off that of lattice 0) and is covered by whole tiles, listed
// lattice by lattice, row by row. A CTA then finds its tile, and the tile it
// prefetches, by arithmetic on list indices instead of loading records
// first (a dependent round trip to memory before its loads can go out).
// G.tiles_x == 0: read the record.
template <typename T, int TX, int TY>
__device__ __forceinline__ void tile_at(const StepArgs<T>& A, const TileGrid& G, int b, Tile& t, Geom& g) {
    if (G.tiles_x > 0) {
        const int lat = div_magic(b, G.m_lat, G.s_lat);
        const int r = b - lat * G.tiles_per_lat;
        const int row = div_magic(r, G.m_x, G.s_x);
        t = Tile{lat, (r - row * G.tiles_x) * TX, row * TY, 1};
        g = G.g0;
        g.f_off += (long long)lat * G.lat_stride;
    } else {
        t = A.tg[b].t;
        g = A.tg[b].g;
    }
}


// The prefetch leads the reads by about DRAM latency x bandwidth under load
// (about 1 us x 6.7 TB/s on GB300), whatever the tile shape: the distance in
// tiles that keeps that many bytes of later tiles' reads on their way.
// Measured on four workloads larger than L2 with four tile shapes, the best
// leads hold 5.5-7.5 MB; leads of 2.5-3.5 MB, or of 14 MB and more, were
// 4-18% slower on the 4096^2 lattice.
constexpr long long kPrefetchLeadBytes = 7ll << 20;
inline int prefetch_lead_tiles(int tile_read_bytes) {
    return (int)((kPrefetchLeadBytes + tile_read_bytes - 1) / tile_read_bytes);
}

// L2 prefetch of the tile that the CTA blockIdx.x + ahead takes (CTAs start
// in about index order): DRAM streams its populations while this CTA and the
// ones between compute, and that CTA finds them in L2. The last `ahead` CTAs
// prefetch the first tiles of the next step instead, so that its first wave
// finds its data in L2 too. Only for workloads
// larger than L2; where the step's data stays in L2 from one step to the next
// the prefetches only add requests (measured 2-5% slower). The tile's rows of the nine planes are TX * sizeof(T) bytes
// each; thread t takes the 128-byte lines t, t + NT, ... (at most PF of them).
// Rows past the lattice's last one are left out. The addresses are computed
// before the CTA's own pulls and the prefetches issued after them, so that
// the own loads go out first.
struct NoAhead {
    __device__ __forceinline__ void issue() const {}
};
template <typename T, int TX, int TY, int NT, bool GRID>
struct AheadLines {
    static constexpr int kLinesPerRow = TX * (int)sizeof(T) / 128;
    static constexpr int kLines = 9 * TY * kLinesPerRow;
    static constexpr int PF = (kLines + NT - 1) / NT;
    const char* p[PF];
    __device__ __forceinline__ void plan(const StepArgs<T>& A, const TileGrid& G) {
        static_assert(TX * sizeof(T) % 128 == 0, "tile rows are whole lines");
#pragma unroll
        for (int k = 0; k < PF; ++k) p[k] = nullptr;
        if (A.ahead <= 0) return;
        const int n = (int)gridDim.x;
        int next = (int)blockIdx.x + A.ahead;
        const T* base = A.fin;
        if (next >= n) {
            // the last CTAs of the launch: the first tiles of the next step,
            // which reads what this step writes (those tiles' rows were
            // written by the first CTAs of this launch, long finished). A
            // hint only: if no such step follows, nothing reads them.
            next -= n;
            base = A.fout;
            if (next >= n) return;
        }
        Tile t;
        Geom g;
        if constexpr (GRID) {
            tile_at<T, TX, TY>(A, G, next, t, g);
        } else {
            t = A.tg[next].t;
            g = A.tg[next].g;
        }
        const int tid = threadIdx.y * TX + threadIdx.x;
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const int line = tid + k * NT;
            const int a = line / (TY * kLinesPerRow);
            const int rem = line - a * (TY * kLinesPerRow);
            const int r = rem / kLinesPerRow, part = rem - r * kLinesPerRow;
            if (line < kLines && t.y0 + r < g.ny)
                p[k] = (const char*)(base + g.f_off + a * g.plane + node_index(g, t.x0, t.y0 + r)) + 128 * part;
        }
    }
    __device__ __forceinline__ void issue() const {
#pragma unroll
        for (int k = 0; k < PF; ++k)
            if (p[k] != nullptr) asm volatile("prefetch.global.L2 [%0];" ::"l"(p[k]));
    }
};

// ---- FP32 node math shared by the plain-load and the TMA kernels: nodes are
// processed in pairs (paired FP32 instructions) when a thread owns an even
// number of them, one at a time otherwise, with bitwise equal results.

// drho, rho, psi of a thread's RY own nodes; a node that is not live reads as
// density rho_ref and gets the solid/absent sentinel psi = -1.
template <int RY>
__device__ __forceinline__ void f32_rho_psi(const float (&f)[RY][9], const bool (&live)[RY], float rho_ref,
                                            const Phys<float>& P, unsigned& flag, float (&drho)[RY],
                                            float (&rho)[RY], float (&psi)[RY]) {
    if constexpr (RY % 2 == 0) {
#pragma unroll
        for (int r = 0; r < RY; r += 2) {
            F2 v[9];
#pragma unroll
            for (int a = 0; a < 9; ++a)
                v[a].v = make_float2(live[r] ? f[r][a] : 0.0f, live[r + 1] ? f[r + 1][a] : 0.0f);
            const F2 d = vsum9(v);
            const F2 rh = splat<F2>(rho_ref) + d;
            const F2 ps = vpsi_any(rh, P, flag);
            drho[r] = d.v.x;
            drho[r + 1] = d.v.y;
            rho[r] = rh.v.x;
            rho[r + 1] = rh.v.y;
            psi[r] = live[r] ? ps.v.x : -1.0f;
            psi[r + 1] = live[r + 1] ? ps.v.y : -1.0f;
        }
    } else {
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            F1 v[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) v[a].v = live[r] ? f[r][a] : 0.0f;
            const F1 d = vsum9(v);
            const F1 rh = splat<F1>(rho_ref) + d;
            const F1 ps = vpsi_any(rh, P, flag);
            drho[r] = d.v;
            rho[r] = rh.v;
            psi[r] = live[r] ? ps.v : -1.0f;
        }
    }
}

// psi of one halo cell from its pulled populations (ANY: every EOS kind;
// else the Carnahan-Starling form the fast paths are restricted to)
template <bool ANY = true>
__device__ __forceinline__ float f32_halo_psi(const float (&fh)[9], float rho_ref, const Phys<float>& P,
                                              unsigned& flag) {
    F1 v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a].v = fh[a];
    const F1 rho = splat<F1>(rho_ref) + vsum9(v);
    if constexpr (ANY)
        return vpsi_any(rho, P, flag).v;
    else
        return vpsi(rho, P, flag).v;
}

// psi of the 8 neighbours of the node at s_psi index c (row stride SW), with
// a solid neighbour (sentinel < 0) replaced by the node's own psi
template <int SW>
__device__ __forceinline__ void f32_neighbours(const float* s_psi, int c, float own, bool walls, float (&nb)[8]) {
    nb[0] = s_psi[c + 1];
    nb[1] = s_psi[c + SW];
    nb[2] = s_psi[c - 1];
    nb[3] = s_psi[c - SW];
    nb[4] = s_psi[c + SW + 1];
    nb[5] = s_psi[c + SW - 1];
    nb[6] = s_psi[c - SW - 1];
    nb[7] = s_psi[c - SW + 1];
    if (walls) {
#pragma unroll
        for (int k = 0; k < 8; ++k) nb[k] = nb[k] < 0.0f ? own : nb[k];
    }
}

// Force (Eq. 7), collision (Eq. 3) and store of the thread's RY own nodes.
// (lx, ly0): tile-local position of the first node; s_psi the psi tile with
// a one-cell frame (row stride SW); x, y0: lattice position.
template <int RY, int SW>
__device__ __forceinline__ void f32_collide_store(float (&f)[RY][9], const bool (&live)[RY],
                                                  const float (&drho)[RY], const float (&rho)[RY],
                                                  const float (&psi)[RY], const float* s_psi, int lx, int ly0,
                                                  bool walls, const Phys<float>& P, float* fo, const Geom& g,
                                                  int x, int y0) {
    const float mG = -P.G;
    const float G2 = __fmul_rn(P.G, P.G);
    if constexpr (RY % 2 == 0) {
#pragma unroll
        for (int r = 0; r < RY; r += 2) {
            const bool do0 = live[r] && y0 + r < g.ny;
            const bool do1 = live[r + 1] && y0 + r + 1 < g.ny;
            if (!(do0 || do1)) continue;
            const int c0 = (ly0 + r + 1) * SW + (lx + 1);
            float n0[8], n1[8];
            f32_neighbours<SW>(s_psi, c0, psi[r], walls, n0);
            f32_neighbours<SW>(s_psi, c0 + SW, psi[r + 1], walls, n1);
            F2 nb[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) nb[k].v = make_float2(n0[k], n1[k]);
            F2 gx, gy;
            vforce_sum(nb[0], nb[1], nb[2], nb[3], nb[4], nb[5], nb[6], nb[7], gx, gy);
            const F2 ps = {make_float2(psi[r], psi[r + 1])};
            const F2 mGpsi = splat<F2>(mG) * ps;
            const F2 Fx = mGpsi * gx, Fy = mGpsi * gy;
            const F2 g2G2 = splat<F2>(G2) * vfma(gx, gx, gy * gy);
            F2 v[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) v[a].v = make_float2(f[r][a], f[r + 1][a]);
            vcollide(v, F2{make_float2(rho[r], rho[r + 1])}, F2{make_float2(drho[r], drho[r + 1])}, Fx, Fy,
                     g2G2, P);
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                f[r][a] = v[a].v.x;
                f[r + 1][a] = v[a].v.y;
            }
            if (do0) store_node<float>(fo, g, x, y0 + r, f[r]);
            if (do1) store_node<float>(fo, g, x, y0 + r + 1, f[r + 1]);
        }
    } else {
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            if (!(live[r] && y0 + r < g.ny)) continue;
            const int c = (ly0 + r + 1) * SW + (lx + 1);
            float n[8];
            f32_neighbours<SW>(s_psi, c, psi[r], walls, n);
            F1 nb[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) nb[k].v = n[k];
            F1 gx, gy;
            vforce_sum(nb[0], nb[1], nb[2], nb[3], nb[4], nb[5], nb[6], nb[7], gx, gy);
            const F1 mGpsi = splat<F1>(mG) * F1{psi[r]};
            const F1 Fx = mGpsi * gx, Fy = mGpsi * gy;
            const F1 g2G2 = splat<F1>(G2) * vfma(gx, gx, gy * gy);
            F1 v[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) v[a].v = f[r][a];
            vcollide(v, F1{rho[r]}, F1{drho[r]}, Fx, Fy, g2G2, P);
#pragma unroll
            for (int a = 0; a < 9; ++a) f[r][a] = v[a].v;
            store_node<float>(fo, g, x, y0 + r, f[r]);
        }
    }
}

// ---- FP32 fast path: a tile that lies wholly inside a lattice of at least
// 4 x 4 nodes with no solid cell in the tile or its two-cell frame (every
// tile of a wall-free lattice). Every own node and halo cell is fluid, so there
// are no liveness tests; a thread's nodes stay in register pairs (F2) from
// the loads to the stores, and only tiles within two cells of a lattice edge
// compute wrapped pull offsets. The arithmetic is that of the general path
// operation for operation, so both give bitwise the same result.

// the nine pulled populations of the vertically adjacent nodes at stored
// indices c and c + pitch, as pairs (no walls, no wrap: every source node
// lies inside the lattice)
__device__ __forceinline__ void pull_pair(const float* __restrict__ fin, int plane, int pitch, int c, F2 f[9]) {
    const int np = 9 * plane;
    auto ld2 = [&](int i) { return F2{make_float2(ld_pop(fin, i, np), ld_pop(fin, i + pitch, np))}; };
    f[0] = ld2(c);
    f[1] = ld2(1 * plane + c - 1);
    f[2] = ld2(2 * plane + c - pitch);
    f[3] = ld2(3 * plane + c + 1);
    f[4] = ld2(4 * plane + c + pitch);
    f[5] = ld2(5 * plane + c - pitch - 1);
    f[6] = ld2(6 * plane + c - pitch + 1);
    f[7] = ld2(7 * plane + c + pitch + 1);
    f[8] = ld2(8 * plane + c + pitch - 1);
}

// pull_pair for a pair at a lattice edge: the first node at stored index c
// (column x, row y), the second one row below it (y + 1 < ny); dxm, dxp are
// the offsets to columns x - 1 and x + 1, rm the offset from row y to row
// y - 1 and rp2 the one from row y + 1 to row y + 2, each periodic (nbr_of).
__device__ __forceinline__ void pull_pair_wrap(const float* __restrict__ fin, int plane, int pitch, int c,
                                               int dxm, int dxp, int rm, int rp2, F2 f[9]) {
    const int np = 9 * plane;
    auto ld2 = [&](int i0, int i1) { return F2{make_float2(ld_pop(fin, i0, np), ld_pop(fin, i1, np))}; };
    const int d = c + pitch;  // the second node
    f[0] = ld2(c, d);
    f[1] = ld2(plane + c + dxm, plane + d + dxm);
    f[2] = ld2(2 * plane + c + rm, 2 * plane + c);
    f[3] = ld2(3 * plane + c + dxp, 3 * plane + d + dxp);
    f[4] = ld2(4 * plane + d, 4 * plane + d + rp2);
    f[5] = ld2(5 * plane + c + rm + dxm, 5 * plane + c + dxm);
    f[6] = ld2(6 * plane + c + rm + dxp, 6 * plane + c + dxp);
    f[7] = ld2(7 * plane + d + dxp, 7 * plane + d + rp2 + dxp);
    f[8] = ld2(8 * plane + d + dxm, 8 * plane + d + rp2 + dxm);
}

// Force (Eq. 7), collision (Eq. 3) and store of the node pair in tile-local
// column lx, rows ly and ly + 1 (psi tile s_psi with a one-cell frame, row
// stride SW), stored index cs of the first node.
template <int SW>
__device__ __forceinline__ void f32_pair_finish(F2 (&f)[9], F2 rho, F2 drho, F2 psi, const float* s_psi, int lx,
                                                int ly, const Phys<float>& P, float* __restrict__ fo, int cs,
                                                int plane, int pitch) {
    const int c = (ly + 1) * SW + lx + 1;
    auto nb2 = [&](int o) { return F2{make_float2(s_psi[c + o], s_psi[c + SW + o])}; };
    F2 gx, gy;
    vforce_sum(nb2(1), nb2(SW), nb2(-1), nb2(-SW), nb2(SW + 1), nb2(SW - 1), nb2(-SW - 1), nb2(-SW + 1), gx, gy);
    const F2 mGpsi = splat<F2>(-P.G) * psi;
    const F2 Fx = mGpsi * gx, Fy = mGpsi * gy;
    const F2 g2G2 = splat<F2>(__fmul_rn(P.G, P.G)) * vfma(gx, gx, gy * gy);
    vcollide(f, rho, drho, Fx, Fy, g2G2, P);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        st_pop(fo, a * plane + cs, 9 * plane, f[a].v.x);
        st_pop(fo, a * plane + cs + pitch, 9 * plane, f[a].v.y);
    }
}

// Position (cx, cy) in the psi tile (SW x SH, one-cell frame around a
// TX x TY tile) of halo ring cell h: top row, bottom row, then the left and
// right columns alternately.
template <int SW, int SH>
__device__ __forceinline__ void halo_ring_cell(int h, int& cx, int& cy) {
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
}

template <int TX, int TYT, int RY, typename PF>
__device__ __forceinline__ void f32_tile_fast(const StepArgs<float>& A, const Tile& tile, const Geom& g,
                                              const Phys<float>& P, float* s_psi, const PF& ahead) {
    static_assert(RY % 2 == 0, "the fast path pairs nodes");
    constexpr int TY = TYT * RY;
    constexpr int SW = TX + 2;
    constexpr int SH = TY + 2;
    constexpr int NT = TX * TYT;
    constexpr int NH = 2 * SW + 2 * TY;
    constexpr int NHT = (NH + NT - 1) / NT;
    constexpr int NP = RY / 2;
    const float* __restrict__ fin = A.fin + g.f_off;
    const int plane = (int)g.plane, pitch = g.pitch;
    const float rho_ref = P.rho_ref;
    unsigned flag = 0;
    const int lx = threadIdx.x, ly0 = threadIdx.y * RY;
    const int x = tile.x0 + lx, y0 = tile.y0 + ly0;
    const int c0 = node_index(g, x, y0);

    // a tile within two cells of an edge has pulls (of its nodes or of its
    // halo ring) that cross it; the others use fixed offsets only
    const bool edge = tile.x0 < 2 || tile.x0 + TX > g.nx - 2 || tile.y0 < 2 || tile.y0 + TY > g.ny - 2;
    F2 f[NP][9];
    if (edge) {
        const int dxm = x == 0 ? g.nx - 1 : -1;
        const int dxp = x == g.nx - 1 ? 1 - g.nx : 1;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int y = y0 + 2 * p;
            const int rm = y == 0 ? (g.ny - 1) * pitch : -pitch;
            const int rp2 = y + 1 == g.ny - 1 ? (1 - g.ny) * pitch : pitch;
            pull_pair_wrap(fin, plane, pitch, c0 + 2 * p * pitch, dxm, dxp, rm, rp2, f[p]);
        }
    } else {
#pragma unroll
        for (int p = 0; p < NP; ++p) pull_pair(fin, plane, pitch, c0 + 2 * p * pitch, f[p]);
    }
    ahead.issue();

    // halo ring: psi only
    float ph[NHT];
    int hc[NHT];
    const int tid = threadIdx.y * TX + threadIdx.x;
#pragma unroll
    for (int k = 0; k < NHT; ++k) {
        const int h = tid + k * NT;
        hc[k] = -1;
        if (h < NH) {
            int cx, cy;
            halo_ring_cell<SW, SH>(h, cx, cy);
            hc[k] = cy * SW + cx;
            const int hx = tile.x0 - 1 + cx, hy = tile.y0 - 1 + cy;
            float fh[9];
            if (edge)
                pull_node<float>(fin, nullptr, plane, nbr_of(g.nx, g.ny, pitch, hx, hy), fh);
            else
                pull_inner<float>(fin, plane, pitch, node_index(g, hx, hy), fh);
            ph[k] = f32_halo_psi<false>(fh, rho_ref, P, flag);
        }
    }

    // own nodes: density and psi
    F2 drho[NP], rho[NP], psi[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        drho[p] = vsum9(f[p]);
        rho[p] = splat<F2>(rho_ref) + drho[p];
        psi[p] = vpsi(rho[p], P, flag);
        s_psi[(ly0 + 2 * p + 1) * SW + lx + 1] = psi[p].v.x;
        s_psi[(ly0 + 2 * p + 2) * SW + lx + 1] = psi[p].v.y;
    }
#pragma unroll
    for (int k = 0; k < NHT; ++k)
        if (hc[k] >= 0) s_psi[hc[k]] = ph[k];
    __syncthreads();
    if (flag) atomicOr(&A.status[tile.lat], flag);

    float* __restrict__ fo = A.fout + g.f_off;
#pragma unroll
    for (int p = 0; p < NP; ++p)
        f32_pair_finish<SW>(f[p], rho[p], drho[p], psi[p], s_psi, lx, ly0 + 2 * p, P, fo, c0 + 2 * p * pitch,
                            plane, pitch);
}

// One tile by the general path (any tile: partial, walled, tiny lattices).
// OPEN: the batch may hold lattices open in x (x-slabs), whose pulls across
// the x edges read the frame instead of wrapping; instantiated apart, so
// that the kernels of ordinary batches compile as if slabs did not exist.
template <typename T, int TX, int TYT, int RY, bool OPEN, typename PF>
__device__ __forceinline__ void tile_general(const StepArgs<T>& A, const Tile& tile, const Geom& g,
                                             const Phys<T>& P, T* s_psi, const PF& ahead) {
    constexpr int TY = TYT * RY;
    constexpr int SW = TX + 2;
    constexpr int SH = TY + 2;
    constexpr int NT = TX * TYT;
    constexpr int NH = 2 * SW + 2 * TY;  // halo ring cells
    const T* __restrict__ fin = A.fin + g.f_off;
    const uint8_t* __restrict__ mask = geom_mask(g) ? A.mask + g.mask_off : nullptr;
    const int plane = (int)g.plane;
    const int nx = g.nx, ny = g.ny, pitch = g.pitch;
    const T rho_ref = P.rho_ref;
    unsigned flag = 0;

    // ---- own nodes: column x, rows y0 .. y0 + RY - 1. Of the cells past the
    // last node (a tile overhanging the lattice) only x = nx and y = ny are
    // pulled: they stand for nodes 0 (periodic), whose psi the last nodes'
    // forces need.
    const int lx = threadIdx.x;
    const int x = tile.x0 + lx;
    const int y0 = tile.y0 + threadIdx.y * RY;
    T f[RY][9];
    bool live[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int y = y0 + r;
        live[r] = (x <= nx) && (y <= ny);
        if (live[r])
            live[r] = !pull_node<T>(fin, mask, plane, OPEN ? nbr_geom(g, x, y) : nbr_of(nx, ny, pitch, x, y), f[r]);
    }
    ahead.issue();

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
                !pull_node<T>(fin, mask, plane, OPEN ? nbr_geom(g, hx, hy) : nbr_of(nx, ny, pitch, hx, hy), fh)) {
                if constexpr (std::is_same<T, float>::value)
                    ph[k] = f32_halo_psi(fh, rho_ref, P, flag);
                else
                    ph[k] = psi_of(rho_ref + sum9(fh), P, flag);
            }
        }
    }

    // ---- own nodes: density and psi
    T drho[RY], rho[RY], psi[RY];
    if constexpr (std::is_same<T, float>::value) {
        f32_rho_psi<RY>(f, live, rho_ref, P, flag, drho, rho, psi);
    } else {
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
        }
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) s_psi[(threadIdx.y * RY + r + 1) * SW + (lx + 1)] = psi[r];
#pragma unroll
    for (int k = 0; k < (NH + NT - 1) / NT; ++k)
        if (hc[k] >= 0) s_psi[hc[k]] = ph[k];
    __syncthreads();

    if (flag) atomicOr(&A.status[tile.lat], flag);
    if (x >= nx) return;

    T* __restrict__ fo = A.fout + g.f_off;
    if constexpr (std::is_same<T, float>::value) {
        f32_collide_store<RY, SW>(f, live, drho, rho, psi, s_psi, lx, threadIdx.y * RY, mask != nullptr, P, fo, g,
                                  x, y0);
    } else {
        const T mG = -P.G;
        const T G2 = P.G * P.G;
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int y = y0 + r;
            if (y >= ny || !live[r]) continue;
            // ---- force, Eq. 7
            const int c = (threadIdx.y * RY + r + 1) * SW + (lx + 1);
            T gx, gy;
            force_sum<T>(mask != nullptr, psi[r], s_psi[c + 1], s_psi[c + SW], s_psi[c - 1], s_psi[c - SW],
                         s_psi[c + SW + 1], s_psi[c + SW - 1], s_psi[c - SW - 1], s_psi[c - SW + 1], gx, gy);
            const T Fx = mG * psi[r] * gx;
            const T Fy = mG * psi[r] * gy;
            // ---- collision, Eq. 3
            collide<T>(f[r], rho[r], drho[r], Fx, Fy, G2 * (gx * gx + gy * gy), P);
            // ---- store f*
            store_node<T>(fo, g, x, y, f[r]);
        }
    }
}

// MINB: minimum resident CTAs per SM the register allocation must allow
// (the register cap is 65536 / (MINB * TX * TYT) per thread). One CTA per
// tile; full tiles of wall-free lattices take the FP32 fast path (an
// x-slab's tiles along its cuts are never marked clear). OPEN: see
// tile_general.
// GRIDARG: the regular tile grid as a trailing argument (only the shapes
// that use it take one, so the others keep their argument layout).
template <typename T, int TX, int TYT, int RY, int MINB, bool TABLE, bool OPEN = false, typename... GRIDARG>
__global__ void __launch_bounds__(TX * TYT, MINB)
    step_kernel(StepArgs<T> A, const __grid_constant__ TableOf<T, TABLE> PT, const GRIDARG... grid_arg) {
    constexpr int TY = TYT * RY;
    constexpr int SW = TX + 2;
    constexpr int SH = TY + 2;
    __shared__ T s_psi[SH * SW];
#ifdef LBM_DEBUG
    // debug builds poison the psi tile, so a cell that no thread writes shows
    // up as NaN in the result
    for (int i = threadIdx.y * TX + threadIdx.x; i < SH * SW; i += TX * TYT) s_psi[i] = T(NAN);
    __syncthreads();
#endif

    // The regular-grid mapping (tile_at) is compiled into the FP32
    // shapes of four nodes per thread only: there it measured 6% faster on a
    // 4096^2 lattice, in the two-node shapes 4% slower (same-box A/B).
    constexpr bool GRID = std::is_same<T, float>::value && RY == 4;
    static_assert(sizeof...(GRIDARG) == (GRID ? 1 : 0), "the grid shapes take a TileGrid, the others none");
    TileGrid G{};
    if constexpr (GRID) G = (grid_arg, ...);
    const bool on_grid = GRID && G.tiles_x > 0;
    // CTA b asks L2 for line b of the tile records, so that the CTAs of
    // later waves find theirs there instead of in DRAM
    if (!on_grid && threadIdx.x == 0 && threadIdx.y == 0) {
        const int nl = (int)((gridDim.x * sizeof(TileGeom) + 127) / 128);
        if ((int)blockIdx.x < nl)
            asm volatile("prefetch.global.L2 [%0];" ::"l"((const char*)A.tg + 128 * (size_t)blockIdx.x));
    }
    Tile tile;
    Geom g;
    if constexpr (GRID) {
        tile_at<T, TX, TY>(A, G, (int)blockIdx.x, tile, g);
    } else {
        tile = A.tg[blockIdx.x].t;
        g = A.tg[blockIdx.x].g;  // independent of the tile load
    }
    // restrict: the stores to fout cannot alias the parameters, so they need
    // not be reloaded after every store
    const Phys<T>* __restrict__ Pp;
    if constexpr (TABLE)
        Pp = &PT.p[tile.lat];
    else
        Pp = A.phys + tile.lat;
    const Phys<T>& P = *Pp;
    auto run = [&](const auto& ahead) {
        if constexpr (std::is_same<T, float>::value && RY % 2 == 0) {
            if (tile.clear && tile.x0 + TX <= g.nx && tile.y0 + TY <= g.ny && g.nx >= 4 && g.ny >= 4 &&
                P.eos == EOS_CS) {
                f32_tile_fast<TX, TYT, RY>(A, tile, g, P, s_psi, ahead);
                return;
            }
        }
        tile_general<T, TX, TYT, RY, OPEN>(A, tile, g, P, s_psi, ahead);
    };
    if constexpr (std::is_same<T, float>::value) {
        AheadLines<T, TX, TY, TX * TYT, GRID> ahead;
        ahead.plan(A, G);
        run(ahead);
    } else {
        run(NoAhead{});  // FP64 storage is bound by the FP64 units, not by DRAM latency
    }
}

}  // namespace lbm
