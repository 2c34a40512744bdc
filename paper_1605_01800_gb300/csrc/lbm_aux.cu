// Non-hot kernels of the library: initial state, macroscopic read-out and the
// FP64 mass and momentum reductions. All arithmetic here is FP64.
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
// With u = 0 (ux, uy null) f_eq_b = w_b rho, and the stored deviation is
// w_b (rho - rho_ref). Invalid input (a fluid density that is not finite and
// > 0, a non-finite velocity) sets bad[lat] = gen: `bad` is the host's
// page-locked flag array, mapped, and gen identifies the host call, so the
// flags need no clearing and no copy back. In-place storage: the swapped
// layout keeps the same values in the opposite planes; the natural layout
// holds f_eq of the node itself in its own planes.
// Density-only init (u = 0) of two-buffer storage and the swapped layout,
// one CTA per 32 x 8 tile. Each stored value is w_b (rho - rho_ref) of the
// node it streams into, and w takes three values (4/9, 1/9, 1/36), so the
// tile and its one-cell frame get their deviation and its three products
// once per cell, in FP64, rounded to the storage type, in shared memory; a
// node's nine values are read from there. The operations are those of
// init_kernel (the FP64 difference, the FP64 product, one rounding), so the
// result is bitwise the same at a third of the FP64 operations.
constexpr int kInitTX = 32, kInitTY = 8;
__device__ __forceinline__ int weight_class(int b) { return b == 0 ? 0 : (b < 5 ? 1 : 2); }
template <typename T>
__global__ void __launch_bounds__(kInitTX * kInitTY, 4)
    init_rho_kernel(const Geom* __restrict__ geoms, const Phys<double>* __restrict__ phys, int lat0,
                    const double* __restrict__ rho, const uint8_t* __restrict__ mask_base, T* __restrict__ f_base,
                    unsigned* __restrict__ bad, unsigned gen, int layout) {
    __shared__ T wd[3][kInitTY + 2][kInitTX + 2];  // (T)(w * (rho - rho_ref)) for w = 4/9, 1/9, 1/36
    const int lat = lat0 + blockIdx.y;
    const Geom g = geoms[lat];
    const double rho_ref = phys[lat].rho_ref;
    const uint8_t* mask = geom_mask(g) ? mask_base + g.mask_off : nullptr;
    T* f = f_base + g.f_off;
    rho += g.node_off;
    const int tiles_x = (g.nx + kInitTX - 1) / kInitTX;
    const int tiles = tiles_x * ((g.ny + kInitTY - 1) / kInitTY);
    const int tid = threadIdx.y * kInitTX + threadIdx.x;
    unsigned invalid = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {  // uniform over the CTA
        const int x0 = (t % tiles_x) * kInitTX, y0 = (t / tiles_x) * kInitTY;
        for (int k = tid; k < (kInitTX + 2) * (kInitTY + 2); k += kInitTX * kInitTY) {
            const int cy = k / (kInitTX + 2), cx = k - cy * (kInitTX + 2);
            // periodic images (a full modulo: a lattice may be narrower or
            // lower than the tile); a cell past the lattice's end is only
            // read by the nodes it neighbours periodically
            const int x = wrap_index(x0 - 1 + cx, g.nx), y = wrap_index(y0 - 1 + cy, g.ny);
            const double dd = rho[y * g.nx + x] - rho_ref;
            wd[0][cy][cx] = (T)(kWeq[0] * dd);
            wd[1][cy][cx] = (T)(kWeq[1] * dd);
            wd[2][cy][cx] = (T)(kWeq[5] * dd);
        }
        __syncthreads();
        const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
        if (x < g.nx && y < g.ny) {
            T out[9];
            if (is_solid(mask, g, x, y)) {
                for (int b = 0; b < 9; ++b) out[b] = T(0);
            } else {
                const double r = rho[y * g.nx + x];
                if (!(isfinite(r) && r > 0.0)) invalid = 1;
#pragma unroll
                for (int b = 0; b < 9; ++b) {
                    int xt = x + kEx[b], yt = y + kEy[b];
                    xt = xt < 0 ? xt + g.nx : (xt >= g.nx ? xt - g.nx : xt);
                    yt = yt < 0 ? yt + g.ny : (yt >= g.ny ? yt - g.ny : yt);
                    // a reflected link stores the node's own value, with the
                    // weight of the same class
                    const bool back = is_solid(mask, g, xt, yt);
                    const int sy = back ? threadIdx.y + 1 : threadIdx.y + 1 + kEy[b];
                    const int sx = back ? threadIdx.x + 1 : threadIdx.x + 1 + kEx[b];
                    const T v = wd[weight_class(b)][sy][sx];
                    if (layout == kLayoutSwapped)  // compile-time indices: out stays in registers
                        out[opp(b)] = v;
                    else
                        out[b] = v;
                }
            }
            store_node<T>(f, g, x, y, out);
        }
        __syncthreads();
    }
    if (invalid) bad[lat] = gen;
}

template <typename T>
__global__ void init_kernel(const Geom* __restrict__ geoms, const Phys<double>* __restrict__ phys,
                            int lat0, const double* __restrict__ rho, const double* __restrict__ ux,
                            const double* __restrict__ uy, const uint8_t* __restrict__ mask_base,
                            T* __restrict__ f_base, unsigned* __restrict__ bad, unsigned gen, int layout) {
    const int lat = lat0 + blockIdx.y;
    const Geom g = geoms[lat];
    const double rho_ref = phys[lat].rho_ref;
    const uint8_t* mask = geom_mask(g) ? mask_base + g.mask_off : nullptr;
    T* f = f_base + g.f_off;
    rho += g.node_off;
    if (ux) ux += g.node_off;
    if (uy) uy += g.node_off;
    const int n = g.nx * g.ny;  // < 2^31: 9 stored planes hold fewer than 2^31 elements
    unsigned invalid = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int y = i / g.nx, x = i - y * g.nx;
        T out[9];
        if (is_solid(mask, g, x, y)) {
            for (int b = 0; b < 9; ++b) out[b] = T(0);
            store_node<T>(f, g, x, y, out);
            continue;
        }
        if (!(isfinite(rho[i]) && rho[i] > 0.0)) invalid = 1;
        if ((ux && !isfinite(ux[i])) || (uy && !isfinite(uy[i]))) invalid = 1;
        for (int b = 0; b < 9; ++b) {
            int j = i;
            int bb = b;
            if (layout != kLayoutNatural) {
                int xt = x + kEx[b], yt = y + kEy[b];
                xt = xt < 0 ? xt + g.nx : (xt >= g.nx ? xt - g.nx : xt);
                yt = yt < 0 ? yt + g.ny : (yt >= g.ny ? yt - g.ny : yt);
                const bool back = is_solid(mask, g, xt, yt);
                j = back ? i : yt * g.nx + xt;
                bb = back ? kOpp[b] : b;
            }
            double v;
            if (ux == nullptr && uy == nullptr)
                v = kWeq[bb] * (rho[j] - rho_ref);
            else
                v = feq(bb, rho[j], ux ? ux[j] : 0.0, uy ? uy[j] : 0.0) - kWeq[bb] * rho_ref;
            out[layout == kLayoutSwapped ? kOpp[b] : b] = (T)v;
        }
        store_node<T>(f, g, x, y, out);
    }
    if (invalid) bad[lat] = gen;
}

// Initial state of one x-slab (a lattice open in x): rho/ux/uy hold
// (nx + 2) x ny values, column x + 1 for x = -1 .. nx (the neighbouring
// slabs' edge columns on either side). As init_kernel, with the pulls across
// the x edges taken from those columns instead of wrapping, and with the
// frame columns the first step pulls from filled as well: x = -1 and x = nx
// with every population (the halo ring's nodes there pull some, and read
// others back where a link comes from a solid cell), x = -2 and x = nx + 1
// with the populations pointing into the lattice. Frame entries no pull
// reads are set to 0.
template <typename T>
__global__ void init_open_kernel(Geom g, double rho_ref, const double* __restrict__ rho,
                                 const double* __restrict__ ux, const double* __restrict__ uy,
                                 const uint8_t* __restrict__ mask_base, T* __restrict__ f_base,
                                 unsigned* __restrict__ bad, int lat, unsigned gen) {
    const uint8_t* mask = geom_mask(g) ? mask_base + g.mask_off : nullptr;
    T* f = f_base + g.f_off;
    const int w = g.nx + 2;                 // columns of the input arrays
    const long long n = (long long)(g.nx + 4) * g.ny;   // cells x = -2 .. nx + 1
    unsigned invalid = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % (g.nx + 4)) - 2, y = (int)(i / (g.nx + 4));
        const int c = node_index(g, x, y);
        const bool own = x >= 0 && x < g.nx;
        const bool solid = is_solid(mask, g, x, y);
        if (own || x == -1 || x == g.nx) {
            const long long k = (long long)y * w + x + 1;
            if (!solid && !(isfinite(rho[k]) && rho[k] > 0.0)) invalid = 1;
            if (!solid && ((ux && !isfinite(ux[k])) || (uy && !isfinite(uy[k])))) invalid = 1;
        }
        for (int b = 0; b < 9; ++b) {
            const bool needed = own || x == -1 || x == g.nx || (x == -2 && kEx[b] == 1) ||
                                (x == g.nx + 1 && kEx[b] == -1);
            double v = 0.0;
            const int xt = x + kEx[b], yt = wrap_index(y + kEy[b], g.ny);
            if (needed && !solid && xt >= -2 && xt <= g.nx + 1) {
                const bool back = is_solid(mask, g, xt, yt);
                // a reflected link is read by the cell itself (only own nodes
                // and the halo columns x = -1, nx pull); a plain one by the
                // cell it points to, which must lie in columns -1 .. nx
                if (back ? (x >= -1 && x <= g.nx) : (xt >= -1 && xt <= g.nx)) {
                    const long long j = back ? (long long)y * w + x + 1 : (long long)yt * w + xt + 1;
                    const int bb = back ? kOpp[b] : b;
                    if (ux == nullptr && uy == nullptr)
                        v = kWeq[bb] * (rho[j] - rho_ref);
                    else
                        v = feq(bb, rho[j], ux ? ux[j] : 0.0, uy ? uy[j] : 0.0) - kWeq[bb] * rho_ref;
                }
            }
            if (own || needed) f[b * g.plane + c] = (T)v;
        }
    }
    if (invalid) bad[lat] = gen;
}

// Halo of an x-slab, 12 * ny values of the stored type: what the neighbour
// on `side` (0: left, 1: right) reads from this slab's state, the nine
// populations of the edge column (its halo ring's node there pulls those
// that point away from this slab or along the edge, and reads the others
// back where a link comes from a solid cell), then the three of the next
// column that point away from this slab. pack reads them from this slab's
// state; unpack writes a neighbour's packed halo into this slab's frame
// (side 0: columns -1, -2 from the left neighbour; side 1: columns nx,
// nx + 1 from the right one).
constexpr int kHaloRows = 12;
__constant__ int kHaloOut[2][kHaloRows] = {{0, 1, 2, 3, 4, 5, 6, 7, 8, 3, 6, 7},
                                           {0, 1, 2, 3, 4, 5, 6, 7, 8, 1, 5, 8}};

template <typename T>
__global__ void halo_pack_kernel(Geom g, const T* __restrict__ f_base, int side, T* __restrict__ out) {
    const T* f = f_base + g.f_off;
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= g.ny) return;
    const int x_outer = side == 0 ? 0 : g.nx - 1, x_inner = side == 0 ? 1 : g.nx - 2;
    for (int k = 0; k < kHaloRows; ++k) {
        const int x = k < 9 ? x_outer : x_inner;
        out[(long long)k * g.ny + y] = f[kHaloOut[side][k] * g.plane + node_index(g, x, y)];
    }
}

template <typename T>
__global__ void halo_unpack_kernel(Geom g, T* __restrict__ f_base, int side, const T* __restrict__ in) {
    T* f = f_base + g.f_off;
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= g.ny) return;
    // the neighbour on the left packed its side 1, the one on the right its side 0
    const int from = 1 - side;
    const int x_outer = side == 0 ? -1 : g.nx, x_inner = side == 0 ? -2 : g.nx + 1;
    for (int k = 0; k < kHaloRows; ++k) {
        const int x = k < 9 ? x_outer : x_inner;
        f[kHaloOut[from][k] * g.plane + node_index(g, x, y)] = in[(long long)k * g.ny + y];
    }
}

// Pulled distribution of node (x, y) as stored (f_a - w_a rho_ref, or f_a
// for plain storage), in FP64; false if solid. The density is rho_ref plus
// their sum (the weights sum to 1) and the momentum their first moment (the
// w_a rho_ref parts cancel), so the read-outs need no per-population FMA.
template <typename T>
__device__ __forceinline__ bool pulled_fp64(const Geom& g, const T* f, const uint8_t* mask, int layout, int x,
                                            int y, double out[9]) {
    T tmp[9];
    if (gather_node<T>(layout, f, mask, (int)g.plane, nbr_geom(g, x, y), tmp)) return false;
    for (int a = 0; a < 9; ++a) out[a] = (double)tmp[a];
    return true;
}

__device__ __forceinline__ double psi_fp64(double rho, const Phys<double>& P) {
    unsigned unused = 0;
    return psi_of(rho, P, unused);
}

// Read-out, pass 1: for every cell with x in [-1, nx], y in [-1, ny] (the
// nodes and, in the frame, their periodic neighbours across each edge) the
// pulled distribution gives rho and psi (Eq. 13) in FP64; psi goes to a
// plane in the stored layout (-1 at solid cells), rho and the momentum
// sum_a e_a f_a of the nodes to the output arrays.
template <typename T>
__global__ void moments_psi_kernel(const Geom* __restrict__ geoms, const Phys<double>* __restrict__ phys,
                                   int lat0, const T* __restrict__ f_base, const uint8_t* __restrict__ mask_base,
                                   double* __restrict__ psi_base, double* __restrict__ rho_out,
                                   double* __restrict__ jx_out, double* __restrict__ jy_out, int layout) {
    const int lat = lat0 + blockIdx.y;
    const Geom g = geoms[lat];
    const Phys<double> P = phys[lat];
    const uint8_t* mask = geom_mask(g) ? mask_base + g.mask_off : nullptr;
    const T* f = f_base + g.f_off;
    double* psi_plane = psi_base + g.f_off / 9;  // one plane per lattice, same indexing
    const long long w = g.nx + 2, n = w * (g.ny + 2);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % w) - 1, y = (int)(i / w) - 1;
        double fc[9];
        const int c = node_index(g, x, y);
        if (!pulled_fp64<T>(g, f, mask, layout, x, y, fc)) {
            psi_plane[c] = -1.0;
            if (x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
                const long long o = g.node_off + (long long)y * g.nx + x;
                rho_out[o] = 0.0;
                jx_out[o] = 0.0;
                jy_out[o] = 0.0;
            }
            continue;
        }
        double rho = P.rho_ref, jx = 0.0, jy = 0.0;
        for (int a = 0; a < 9; ++a) {
            rho += fc[a];
            jx += kEx[a] * fc[a];
            jy += kEy[a] * fc[a];
        }
        psi_plane[c] = psi_fp64(rho, P);
        if (x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
            const long long o = g.node_off + (long long)y * g.nx + x;
            rho_out[o] = rho;
            jx_out[o] = jx;
            jy_out[o] = jy;
        }
    }
}

// Read-out of the density alone (when no other moment is asked for): rho of
// every node from its pulled distribution, summed in FP64 in the order of
// moments_psi_kernel (so both give the same value), 0 at solid nodes.
template <typename T>
__global__ void density_kernel(const Geom* __restrict__ geoms, const Phys<double>* __restrict__ phys, int lat0,
                               const T* __restrict__ f_base, const uint8_t* __restrict__ mask_base,
                               double* __restrict__ rho_out, int layout) {
    const int lat = lat0 + blockIdx.y;
    const Geom g = geoms[lat];
    const double rho_ref = phys[lat].rho_ref;
    const uint8_t* mask = geom_mask(g) ? mask_base + g.mask_off : nullptr;
    const T* f = f_base + g.f_off;
    const int n = g.nx * g.ny;  // < 2^31: 9 stored planes hold fewer than 2^31 elements
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int y = i / g.nx, x = i - y * g.nx;
        double fc[9];
        double rho = 0.0;
        if (pulled_fp64<T>(g, f, mask, layout, x, y, fc)) {
            rho = rho_ref;
            for (int a = 0; a < 9; ++a) rho += fc[a];
        }
        rho_out[g.node_off + i] = rho;
    }
}

// Force of Eq. 7 at the fluid node with cell index c and pseudopotential psi,
// from a psi plane with a one-cell frame (negative psi marks a solid cell,
// which takes the node's own psi).
__device__ __forceinline__ void force_fp64(const Geom& g, const Phys<double>& P, const double* psi_plane, int c,
                                           double psi, double& Fx, double& Fy) {
    double gx = 0.0, gy = 0.0;
    for (int a = 1; a < 9; ++a) {
        double pn = psi_plane[c + kEy[a] * g.pitch + kEx[a]];
        pn = pn < 0.0 ? psi : pn;
        const double wa = (a < 5) ? (1.0 / 3.0) : (1.0 / 12.0);
        gx += wa * pn * kEx[a];
        gy += wa * pn * kEy[a];
    }
    Fx = -P.G * psi * gx;
    Fy = -P.G * psi * gy;
}

// Read-out, pass 2: force (Eq. 7, a solid neighbour takes the node's psi),
// velocity (Eq. 6) and pressure (Eq. 10) of every node; ux/uy hold the
// momentum on entry and the velocity on exit.
__global__ void moments_force_kernel(const Geom* __restrict__ geoms, const Phys<double>* __restrict__ phys,
                                     int lat0, const double* __restrict__ psi_base, const double* __restrict__ rho,
                                     double* __restrict__ ux, double* __restrict__ uy, double* __restrict__ p) {
    const int lat = lat0 + blockIdx.y;
    const Geom g = geoms[lat];
    const Phys<double> P = phys[lat];
    const double* psi_plane = psi_base + g.f_off / 9;
    const long long n = (long long)g.nx * g.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)(i / g.nx);
        const long long o = g.node_off + i;
        const int c = node_index(g, x, y);
        const double psi = psi_plane[c];
        if (psi < 0.0) {  // solid node
            ux[o] = 0.0;
            uy[o] = 0.0;
            p[o] = 0.0;
            continue;
        }
        double Fx, Fy;
        force_fp64(g, P, psi_plane, c, psi, Fx, Fy);
        const double r = rho[o];
        ux[o] = (ux[o] + 0.5 * Fx) / r;
        uy[o] = (uy[o] + 0.5 * Fy) / r;
        // Eq. 10: p = rho c_s^2 + G c^2 psi^2 / 2
        p[o] = r * P.cs2 + 0.5 * P.G * psi * psi;
    }
}

// Partial sums: block b adds the post-collision values of the fluid nodes
// i = b*T + t + k*B*T (the stored values of two-buffer storage; in-place
// storage finds them by the layout) in a fixed order, then a fixed tree
// inside the block.
template <typename T>
__global__ void mass_partial_kernel(Geom g, const T* __restrict__ f, const uint8_t* __restrict__ mask,
                                    int layout, double* __restrict__ partials) {
    __shared__ double red[kMassThreads];
    const long long n = (long long)g.nx * g.ny;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)kMassThreads + threadIdx.x; i < n;
         i += (long long)kMassBlocks * kMassThreads) {
        const int x = (int)(i % g.nx), y = (int)(i / g.nx);
        if (is_solid(mask, g, x, y)) continue;
        T fs[9];
        post_collision_node<T>(layout, f, mask, (int)g.plane, nbr_of(g.nx, g.ny, g.pitch, x, y), fs);
        double s = 0.0;
        for (int a = 0; a < 9; ++a) s += (double)fs[a];
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

// Per-lattice totals after moments_psi_kernel (psi plane, j in jx/jy): block
// b of lattice lat0 + blockIdx.y visits the fluid nodes i = b*T + t + k*B*T
// and adds (0) the stored values, in the order of mass_partial_kernel, (1)
// one per node, (2, 3) j + F/2, the numerator of Eq. 6; then the same fixed
// tree as mass_partial_kernel. partials[((lat - lat0)*4 + q)*B + b].
template <typename T>
__global__ void totals_partial_kernel(const Geom* __restrict__ geoms, const Phys<double>* __restrict__ phys,
                                      int lat0, const T* __restrict__ f_base, const uint8_t* __restrict__ mask_base,
                                      const double* __restrict__ psi_base, const double* __restrict__ jx,
                                      const double* __restrict__ jy, int layout, double* __restrict__ partials) {
    __shared__ double red[4][kMassThreads];
    const int lat = lat0 + blockIdx.y;
    const Geom g = geoms[lat];
    const Phys<double> P = phys[lat];
    const uint8_t* mask = geom_mask(g) ? mask_base + g.mask_off : nullptr;
    const T* f = f_base + g.f_off;
    const double* psi_plane = psi_base + g.f_off / 9;
    const long long n = (long long)g.nx * g.ny;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long i = blockIdx.x * (long long)kMassThreads + threadIdx.x; i < n;
         i += (long long)kMassBlocks * kMassThreads) {
        const int x = (int)(i % g.nx), y = (int)(i / g.nx);
        if (is_solid(mask, g, x, y)) continue;
        const long long c = node_index(g, x, y);
        T fs[9];
        post_collision_node<T>(layout, f, mask, (int)g.plane, nbr_of(g.nx, g.ny, g.pitch, x, y), fs);
        double s = 0.0;
        for (int a = 0; a < 9; ++a) s += (double)fs[a];
        acc[0] += s;
        acc[1] += 1.0;
        double Fx, Fy;
        force_fp64(g, P, psi_plane, (int)c, psi_plane[c], Fx, Fy);
        const long long o = g.node_off + i;
        acc[2] += jx[o] + 0.5 * Fx;
        acc[3] += jy[o] + 0.5 * Fy;
    }
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kMassThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4)
        partials[((long long)blockIdx.y * 4 + threadIdx.x) * kMassBlocks + blockIdx.x] = red[threadIdx.x][0];
}

// One thread per lattice: out[3k] = mass (the partial sums in block order
// plus rho_ref times the fluid node count, as mass_final_kernel), out[3k + 1],
// out[3k + 2] = the momentum sums.
__global__ void totals_final_kernel(const double* __restrict__ partials, const Phys<double>* __restrict__ phys,
                                    int lat0, int n_lat, double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_lat) return;
    double s[4];
    for (int q = 0; q < 4; ++q) {
        const double* p = partials + ((long long)k * 4 + q) * kMassBlocks;
        double t = 0.0;
        for (int b = 0; b < kMassBlocks; ++b) t += p[b];
        s[q] = t;
    }
    out[3 * k] = __fma_rn(phys[lat0 + k].rho_ref, s[1], s[0]);
    out[3 * k + 1] = s[2];
    out[3 * k + 2] = s[3];
}

__global__ void mass_final_kernel(const double* __restrict__ partials, double rho_ref,
                                  long long n_fluid, double* out) {
    double s = 0.0;
    for (int b = 0; b < kMassBlocks; ++b) s += partials[b];
    *out = __fma_rn(rho_ref, (double)n_fluid, s);
}

dim3 lattice_grid(long long max_nodes, int n_lat, int threads) {
    long long bx = (max_nodes + threads - 1) / threads;
    if (bx > 4096) bx = 4096;
    if (bx < 1) bx = 1;
    return dim3((unsigned)bx, (unsigned)n_lat);
}

template <typename T>
cudaError_t init_impl(const LaunchSet& L, const double* rho, const double* ux, const double* uy,
                      T* f, unsigned* bad, unsigned gen, cudaStream_t s) {
    if (ux == nullptr && uy == nullptr && L.layout != kLayoutNatural) {
        long long tiles = (L.max_nodes + kInitTX * kInitTY - 1) / (kInitTX * kInitTY) + L.max_extent / 8 + 1;
        if (tiles > 4096) tiles = 4096;
        init_rho_kernel<T><<<dim3((unsigned)tiles, L.n_lat), dim3(kInitTX, kInitTY), 0, s>>>(
            L.geoms, L.phys, L.lat0, rho, L.mask, f, bad, gen, L.layout);
    } else {
        init_kernel<T><<<lattice_grid(L.max_nodes, L.n_lat, 256), 256, 0, s>>>(
            L.geoms, L.phys, L.lat0, rho, ux, uy, L.mask, f, bad, gen, L.layout);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t init_open_impl(const Geom& g, double rho_ref, const double* rho, const double* ux, const double* uy,
                           const uint8_t* mask, T* f, unsigned* bad, int lat, unsigned gen, cudaStream_t s) {
    long long cells = (long long)(g.nx + 4) * g.ny;
    long long blocks = (cells + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    init_open_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(g, rho_ref, rho, ux, uy, mask, f, bad, lat, gen);
    return cudaGetLastError();
}

template <typename T>
cudaError_t halo_impl(const Geom& g, T* f, int side, T* buf, bool pack, cudaStream_t s) {
    const unsigned blocks = (unsigned)((g.ny + 127) / 128);
    if (pack)
        halo_pack_kernel<T><<<blocks, 128, 0, s>>>(g, f, side, buf);
    else
        halo_unpack_kernel<T><<<blocks, 128, 0, s>>>(g, f, side, buf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t moments_impl(const LaunchSet& L, const T* f, double* psi, double* rho, double* ux, double* uy,
                         double* p, cudaStream_t s) {
    // cells of the nodes plus a one-cell frame: (nx + 2)(ny + 2) <= nodes + 2(nx + ny) + 4
    moments_psi_kernel<T><<<lattice_grid(L.max_nodes + 2 * L.max_extent + 4, L.n_lat, 128), 128, 0, s>>>(
        L.geoms, L.phys, L.lat0, f, L.mask, psi, rho, ux, uy, L.layout);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    moments_force_kernel<<<lattice_grid(L.max_nodes, L.n_lat, 128), 128, 0, s>>>(L.geoms, L.phys, L.lat0, psi,
                                                                                 rho, ux, uy, p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t density_impl(const LaunchSet& L, const T* f, double* rho, cudaStream_t s) {
    density_kernel<T><<<lattice_grid(L.max_nodes, L.n_lat, 256), 256, 0, s>>>(L.geoms, L.phys, L.lat0, f, L.mask,
                                                                               rho, L.layout);
    return cudaGetLastError();
}

template <typename T>
cudaError_t totals_impl(const LaunchSet& L, const T* f, double* psi, double* rho, double* jx, double* jy,
                        double* partials, double* out, cudaStream_t s) {
    moments_psi_kernel<T><<<lattice_grid(L.max_nodes + 2 * L.max_extent + 4, L.n_lat, 128), 128, 0, s>>>(
        L.geoms, L.phys, L.lat0, f, L.mask, psi, rho, jx, jy, L.layout);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    totals_partial_kernel<T><<<dim3(kMassBlocks, L.n_lat), kMassThreads, 0, s>>>(L.geoms, L.phys, L.lat0, f, L.mask,
                                                                                psi, jx, jy, L.layout, partials);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    totals_final_kernel<<<(L.n_lat + 127) / 128, 128, 0, s>>>(partials, L.phys, L.lat0, L.n_lat, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mass_impl(const Geom& g, double rho_ref, long long n_fluid, const T* f,
                      const uint8_t* mask, int layout, double* partials, double* out, cudaStream_t s) {
    mass_partial_kernel<T><<<kMassBlocks, kMassThreads, 0, s>>>(g, f + g.f_off, mask, layout, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mass_final_kernel<<<1, 1, 0, s>>>(partials, rho_ref, n_fluid, out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init_f32(const LaunchSet& L, const double* rho, const double* ux,
                            const double* uy, float* f, unsigned* bad, unsigned gen, cudaStream_t s) {
    return init_impl<float>(L, rho, ux, uy, f, bad, gen, s);
}
cudaError_t launch_init_f64(const LaunchSet& L, const double* rho, const double* ux,
                            const double* uy, double* f, unsigned* bad, unsigned gen, cudaStream_t s) {
    return init_impl<double>(L, rho, ux, uy, f, bad, gen, s);
}
cudaError_t launch_init_open_f32(const Geom& g, double rho_ref, const double* rho, const double* ux,
                                 const double* uy, const uint8_t* mask, float* f, unsigned* bad, int lat,
                                 unsigned gen, cudaStream_t s) {
    return init_open_impl<float>(g, rho_ref, rho, ux, uy, mask, f, bad, lat, gen, s);
}
cudaError_t launch_init_open_f64(const Geom& g, double rho_ref, const double* rho, const double* ux,
                                 const double* uy, const uint8_t* mask, double* f, unsigned* bad, int lat,
                                 unsigned gen, cudaStream_t s) {
    return init_open_impl<double>(g, rho_ref, rho, ux, uy, mask, f, bad, lat, gen, s);
}
cudaError_t launch_halo_f32(const Geom& g, float* f, int side, float* buf, bool pack, cudaStream_t s) {
    return halo_impl<float>(g, f, side, buf, pack, s);
}
cudaError_t launch_halo_f64(const Geom& g, double* f, int side, double* buf, bool pack, cudaStream_t s) {
    return halo_impl<double>(g, f, side, buf, pack, s);
}
cudaError_t launch_density_f32(const LaunchSet& L, const float* f, double* rho, cudaStream_t s) {
    return density_impl<float>(L, f, rho, s);
}
cudaError_t launch_density_f64(const LaunchSet& L, const double* f, double* rho, cudaStream_t s) {
    return density_impl<double>(L, f, rho, s);
}

cudaError_t launch_moments_f32(const LaunchSet& L, const float* f, double* psi, double* rho, double* ux,
                               double* uy, double* p, cudaStream_t s) {
    return moments_impl<float>(L, f, psi, rho, ux, uy, p, s);
}
cudaError_t launch_moments_f64(const LaunchSet& L, const double* f, double* psi, double* rho, double* ux,
                               double* uy, double* p, cudaStream_t s) {
    return moments_impl<double>(L, f, psi, rho, ux, uy, p, s);
}
cudaError_t launch_totals_f32(const LaunchSet& L, const float* f, double* psi, double* rho, double* jx,
                              double* jy, double* partials, double* out, cudaStream_t s) {
    return totals_impl<float>(L, f, psi, rho, jx, jy, partials, out, s);
}
cudaError_t launch_totals_f64(const LaunchSet& L, const double* f, double* psi, double* rho, double* jx,
                              double* jy, double* partials, double* out, cudaStream_t s) {
    return totals_impl<double>(L, f, psi, rho, jx, jy, partials, out, s);
}
cudaError_t launch_mass_f32(const Geom& g, double rho_ref, long long n_fluid, const float* f,
                            const uint8_t* mask, int layout, double* partials, double* out, cudaStream_t s) {
    return mass_impl<float>(g, rho_ref, n_fluid, f, mask, layout, partials, out, s);
}
cudaError_t launch_mass_f64(const Geom& g, double rho_ref, long long n_fluid, const double* f,
                            const uint8_t* mask, int layout, double* partials, double* out, cudaStream_t s) {
    return mass_impl<double>(g, rho_ref, n_fluid, f, mask, layout, partials, out, s);
}

}  // namespace lbm
